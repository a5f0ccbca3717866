/*
 * hdg.h -- C ABI of libhdg: the data-parallel hot path of the hybridizable discontinuous
 * Galerkin (HDG) method for variable-coefficient reaction-diffusion on conforming
 * tetrahedral meshes at a fixed polynomial degree k (Fu, Gatica, Sayas, "Matlab tools for
 * HDG in three dimensions", arXiv 1305.1489), on one NVIDIA GB300 (sm_103a).
 *
 * Problem (eq. 1.1):  kappa^-1 q + grad u = 0,  div q + c u = f  in Omega,
 *                     u = u_D on Gamma_D,  -q.nu = g_N.nu on Gamma_N.
 * Unknowns (eq. 1.2): q_h in P_k(K)^3, u_h in P_k(K) per element, u_hat in P_k(e) per face.
 *
 * Conventions shared by every call
 *  - All indices are 0-based.  Host arrays are row-major (C order).
 *  - "device" pointers are CUDA global-memory pointers on the device that was current when
 *    hdg_mesh_create ran; "host" pointers are ordinary CPU memory.
 *  - Element-major layout ("SoA per element"): an array documented [Nelt][Nq] holds the Nq
 *    values of element 0, then of element 1, ...
 *  - Quadrature: volume nodes are the conical Gauss-Jacobi rule with (k+2)^3 nodes (exact
 *    to degree 2k+3); face nodes the (k+2)^2-node rule on each face (eq. 3.1, Section 4).
 *  - Bases: orthonormal hierarchical Dubiner bases, int_K P_i P_j = |K| delta_ij and
 *    int_e D_i D_j = |e| delta_ij (eq. 3.3, Section 4), ordered by degree then (p,q[,r]).
 *  - Global faces are numbered in lexicographic order of their sorted vertex triples; a
 *    face's parametrisation phi_e uses its vertices in ascending order (Section 2).
 *  - Every call returns an hdg_status (0 = success).  No call throws.  On failure the
 *    message of the last error of the calling thread is available from hdg_last_error.
 *  - Work is enqueued on the CUDA stream given to hdg_mesh_create.  Calls returning values
 *    to the host (iteration counts, residuals, status counts) synchronise that stream.
 *  - A mesh handle may be used by one host thread at a time.
 */
#ifndef HDG_H
#define HDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HDG_OK = 0,
  HDG_ERR_ARG = 1,             /* invalid argument (null pointer, size, degree ...)        */
  HDG_ERR_ORIENTATION = 2,     /* an element has det B_K <= 0 (Section 2 requires > 0)     */
  HDG_ERR_NONCONFORMING = 3,   /* a face shared by >2 elements, or a boundary face missing
                                  from both boundary lists, or a listed face not in the mesh */
  HDG_ERR_CUDA = 4,            /* a CUDA runtime call failed                                */
  HDG_ERR_STATE = 5,           /* calls out of order (e.g. solve before assemble)           */
  HDG_ERR_LOCAL_SINGULAR = 6,  /* a local factorisation met a non-positive pivot           */
  HDG_ERR_NOT_CONVERGED = 7,   /* the trace solve hit maxit before the tolerance            */
  HDG_ERR_COEFF = 8,           /* kappa <= 0 or c < 0 or a non-finite coefficient value     */
  HDG_ERR_UNSUPPORTED = 9      /* option not built (e.g. degree outside 0..4)               */
} hdg_status;

typedef enum {
  HDG_FP64 = 0,        /* every operation in IEEE double                                   */
  HDG_MIXED_FP32 = 1,  /* FP32 inner solve with FP64 residuals and refinement (solve only) */
  HDG_DF32 = 2,        /* assembly only: double-float arithmetic (pairs of FP32, ~48-bit
                          significand) on the FP32 pipe; results stored as FP64           */
  HDG_MIXED_BF16 = 3   /* assembly only: the volume masses on the tensor cores from split
                          BF16 operands (FP32-level), the condensation as HDG_DF32       */
} hdg_precision;

typedef struct hdg_mesh hdg_mesh;

typedef struct {
  int64_t nelt, nfc, ndir, nneu, nver;
  int32_t k;      /* polynomial degree                                    */
  int32_t n;      /* d3 = (k+1)(k+2)(k+3)/6, dim P_k(K)                    */
  int32_t d2;     /* (k+1)(k+2)/2, dim P_k(e)                              */
  int32_t m;      /* 4 d2, dim R_k(dK) (local trace space, Section 5)      */
  int32_t n1;     /* d3(k+1), dim P_{k+1}(K) for the postprocess u*        */
  int32_t nq;     /* volume quadrature nodes per element, (k+2)^3          */
  int32_t nf;     /* face quadrature nodes per face, (k+2)^2               */
  int32_t has_convection;
} hdg_mesh_info;

/* Build the expanded mesh (Section 2: faces, facebyele, perm, normals) from the basic one.
 *   coords [nver][3] host f64; elems [nelt][4] host int32, positively oriented;
 *   dir [ndir][3], neu [nneu][3] host int32 vertex triples (any order within a triple).
 *   k in 0..4 (k = 0: the HDG method without convection; batches, the BDM element and
 *   hdg_solve_trace_noalloc need k >= 1).  stream: cudaStream_t to use (NULL = legacy
 *   default stream).
 * The library copies what it needs; the caller's arrays may be freed on return.
 * Every boundary face must be listed exactly once in dir or neu (Gamma = Gamma_D U Gamma_N).
 * Errors: HDG_ERR_ARG, HDG_ERR_ORIENTATION, HDG_ERR_NONCONFORMING, HDG_ERR_CUDA.          */
int hdg_mesh_create(const double* coords, int64_t nver, const int32_t* elems, int64_t nelt,
                    const int32_t* dir, int64_t ndir, const int32_t* neu, int64_t nneu,
                    int k, void* stream, hdg_mesh** out);

/* Release every device and host resource of the handle (NULL is accepted). */
int hdg_mesh_destroy(hdg_mesh* mesh);

/* Sizes of the discrete spaces (host struct filled in). */
int hdg_mesh_get_info(const hdg_mesh* mesh, hdg_mesh_info* info);

/* Expanded-mesh fields, host outputs (any may be NULL):
 *   faces [nfc][4] int32: sorted vertex triple + type (0 interior, 1 Dirichlet, 2 Neumann);
 *   facebyele [nelt][4] int32 (global face of local face l, eq. 2.1 order);
 *   perm [nelt][4] int32 in 1..6 (eq. 2.3).                                               */
int hdg_mesh_get_faces(const hdg_mesh* mesh, int32_t* faces, int32_t* facebyele, int32_t* perm);

/* Quadrature nodes where the caller evaluates the PDE data (eq. 3.4 and eq. 6.2).
 *   X, Y, Z: device f64 [nelt][nq] volume nodes p_q^K = F_K(p_hat_q);
 *   FX, FY, FZ: device f64 [nfc][nf] face nodes q_r^e = phi_e(q_hat_r).
 * Either triple may be NULL.                                                              */
int hdg_quadrature_nodes(hdg_mesh* mesh, double* X, double* Y, double* Z,
                         double* FX, double* FY, double* FZ);

/* PDE coefficients at the volume nodes (device f64, borrowed: they must stay valid until
 * the next hdg_assemble_condense and hdg_postprocess that use them have completed).
 *   kappa [nelt][nq] > 0, c [nelt][nq] >= 0, f [nelt][nq];
 *   beta [3][nelt][nq]: convection field (Section 9, eq. 9.1) or NULL for reaction-diffusion;
 *     when given, hdg_set_face_convection must also be called before assembly;
 *   tau [nelt][4] >= 0 per element face (eq. 4.22), or NULL for tau = 1.
 * With convection the method solves div(q + beta u) + c u = f with the numerical flux
 * q.nu + (beta.nu) u_hat + tau (u - u_hat); tau - beta.nu/2 > 0 and c + div(beta)/2 >= 0
 * are the caller's responsibility (they make the local solves and the trace system
 * well posed).  Positivity of kappa and c is checked in hdg_assemble_condense (HDG_ERR_COEFF). */
int hdg_set_coefficients(hdg_mesh* mesh, const double* kappa, const double* c,
                         const double* beta, const double* f, const double* tau);

/* Element face nodes F_K(q_hat_r^l) (eq. 4.1): X, Y, Z device f64 [nelt][4][nf], the points
 * where the convection field enters the face integrals of Section 9.                     */
int hdg_element_face_nodes(hdg_mesh* mesh, double* X, double* Y, double* Z);

/* Convection field at the element face nodes, beta_f [3][nelt][4][nf] device f64 (borrowed).
 * Used by the face matrices <(beta.nu) D_i, P_j> and <(beta.nu) D_i, D_j> (Section 9).   */
int hdg_set_face_convection(hdg_mesh* mesh, const double* beta_f);

/* Boundary data at the face nodes (device f64, borrowed like the coefficients):
 *   uD [nfc][nf]: u_D at the face nodes (read on Dirichlet faces only), or NULL for u_D = 0;
 *   gN [3][nfc][nf]: the vector field g_N (read on Neumann faces only), or NULL for g_N = 0.
 * Neumann data enter through eq. 6.4 with the outward normal of the face's element.      */
int hdg_set_boundary_data(hdg_mesh* mesh, const double* uD, const double* gN);

/* Per-element assembly of the local blocks and static condensation (Sections 3-5):
 * C^K = A3 A1^-1 A2 + tauDD (eq. 5.5), C_f^K = A3 A1^-1 A_f (eq. 5.6), and the operators of
 * the local recovery (eq. 5.3), into library-owned device memory.
 * precision: HDG_FP64 (native FP64) or HDG_DF32 (double-float on the FP32 pipe, FP64-level
 * accuracy; with convection the non-symmetric Schur complement is factored by a double-float
 * LU without pivoting; at k = 0 it runs the FP64 kernel), or HDG_MIXED_BF16: the volume masses
 * M_{kappa^-1}, M_c and f^K (eq. 3.55-3.56, 4.3) as one tensor-core contraction over all
 * elements (tcgen05, each FP64 operand split into three BF16 parts, the six products above
 * 2^-24 accumulated in FP32; masses and f^K to FP32-level rounding), then the HDG_DF32
 * condensation from them; k >= 1 and the conical rule (HDG_ERR_UNSUPPORTED otherwise); it
 * holds nelt x 4 ceil((n(n+1) + n) / 4) bytes of FP32 masses.  The precision also
 * selects that of hdg_recover and hdg_postprocess until the next assembly.  Synchronises to report
 * HDG_ERR_LOCAL_SINGULAR / HDG_ERR_COEFF (with the count of failing elements in the message). */
int hdg_assemble_condense(hdg_mesh* mesh, int precision);

/* The same assembly from host arrays, with the host -> device copies overlapped with the
 * condensation (Sections 3-5): the library copies the inputs into device buffers of its own
 * (allocated on first use, kept with the mesh), makes them the mesh's coefficients,
 * convection field and boundary data (as hdg_set_coefficients, hdg_set_face_convection and
 * hdg_set_boundary_data would), and with precision HDG_DF32 condenses the elements in
 * `chunks` consecutive ranges (growing by a factor 1.25, so that the first copy, the only one
 * nothing overlaps, is short), each range launched as soon as its inputs have landed while
 * the next range is copied (a second stream and events).  Other precisions copy everything
 * first and run hdg_assemble_condense.  Host arrays in the layouts of the device calls;
 * page-locked (pinned) memory lets the copies run beside the kernels, pageable memory is
 * copied through staging by the driver.  Synchronises; errors as hdg_assemble_condense, and
 * HDG_ERR_ARG for missing kappa, c, f or only one of beta, beta_f.                        */
typedef struct hdg_host_inputs {
  const double *kappa, *c, *f;  /* [nelt][nq] (required)                                    */
  const double *beta, *beta_f;  /* [3][nelt][nq] and [3][nelt][4][nf], both or neither      */
  const double *tau;            /* [nelt][4] or NULL (tau = 1)                               */
  const double *uD, *gN;        /* [nfc][nf] and [3][nfc][nf], each or NULL (as for
                                   hdg_set_boundary_data; both NULL keeps the current data) */
} hdg_host_inputs;
int hdg_assemble_condense_host(hdg_mesh* mesh, int precision, const hdg_host_inputs* in, int chunks);

/* Volume quadrature rule (eq. 3.1; the paper leaves the rule open and remarks that suitable
 * rules are easy to find):
 *   HDG_RULE_CONICAL (default): conical-product Gauss-Jacobi, (k+2)^3 nodes;
 *   HDG_RULE_SYMMETRIC: the fully symmetric Grundmann-Moller rule of the same degree 2k+3 with
 *   C(k+5, 4) nodes (k = 1..4: 15, 35, 70, 126 instead of 27, 64, 125, 216; some weights
 *   negative), which cuts the coefficient data and the direct quadrature sums of the FP64
 *   assembly.  The rule changes the discrete solution by the quadrature error, so it is the
 *   caller's choice, not the autotuner's.
 * Call right after hdg_mesh_create: every array at the volume nodes changes size, so the
 * coefficients are unset (set them again from hdg_quadrature_nodes) and the assembly is
 * invalidated.  The double-float assembly needs the conical rule (its masses are summed by
 * sum factorisation over the conical product): hdg_assemble_condense(HDG_DF32) returns
 * HDG_ERR_UNSUPPORTED with the symmetric rule.  HDG_ERR_ARG for another value.            */
typedef enum { HDG_RULE_CONICAL = 0, HDG_RULE_SYMMETRIC = 1 } hdg_volume_rule;
int hdg_set_volume_rule(hdg_mesh* mesh, int rule);

/* Local method of the next hdg_assemble_condense (Section 9, "BDM"):
 *   HDG_METHOD_HDG (default): the HDG method of eq. 1.2;
 *   HDG_METHOD_BDM: the hybridised Brezzi-Douglas-Marini element, tau = 0 (the tau given to
 *   hdg_set_coefficients is ignored) and u_h in P_{k-1}(K): the degree-k members of the
 *   hierarchical u basis are erased from the local problem (hdg_recover returns them as 0),
 *   q_h stays in P_k(K)^3, everything else (trace solve, recovery, postprocess) unchanged.
 * HDG_ERR_ARG for another value; hdg_assemble_condense returns HDG_ERR_UNSUPPORTED for BDM
 * with convection.                                                                        */
typedef enum { HDG_METHOD_HDG = 0, HDG_METHOD_BDM = 1 } hdg_method;
int hdg_set_method(hdg_mesh* mesh, int method);

/* Copy the condensed local matrices out (tests): C [nelt][m][m] (row-major C^K), Cf [nelt][m]
 * device f64.                                                                              */
int hdg_get_condensed(const hdg_mesh* mesh, double* C, double* Cf);

/* Global trace system H u_hat = F + G_N (eq. 6.5), Dirichlet faces eliminated (Section 6),
 * solved matrix-free element by element with block-Jacobi preconditioned CG (BiCGStab when a
 * convection field is set: the trace matrix is then non-symmetric) to
 *   ||b - H u_hat||_2 <= rtol ||b||_2  (FP64 residual over the free dofs).
 *   precision: HDG_FP64 (plain PCG or BiCGStab) or HDG_MIXED_FP32 (FP32 inner PCG or BiCGStab
 *   iterations, FP64 residuals and refinement; an inner breakdown restarts from the refined
 *   iterate).
 *   x0: device f64 [nfc][d2] initial guess or NULL (zero start); its entries on Dirichlet faces
 *   are ignored (u_hat_D enters through the right-hand side), so a previous uhat is a valid guess.
 *   uhat: device f64 [nfc][d2] output; Dirichlet faces receive u_hat_D of eq. 6.3.
 *   iters, relres: host outputs (may be NULL): iterations (inner iterations for the mixed
 *   path) and the final FP64 relative residual.
 * Returns HDG_ERR_NOT_CONVERGED (with uhat holding the last iterate) when maxit is hit.    */
int hdg_solve_trace(hdg_mesh* mesh, int precision, double rtol, int maxit, const double* x0,
                    double* uhat, int* iters, double* relres);

/* Same solve as hdg_solve_trace with precision HDG_FP64, for callers that cannot allocate
 * device memory when they solve (an application that reserves its whole device-memory budget
 * up front, or a pool-managed framework that forbids allocations after warm-up; cudaMalloc
 * would also synchronise the device).  The paper has no counterpart: this is a deployment
 * variant.  It allocates nothing: every scratch buffer (right-hand side, boundary data,
 * block-Jacobi inverses, Krylov vectors, reduction partials) lives in one file-scope static
 * device array of 11.6 MiB that each GPU loading the library holds until the process exits.
 *   Limit: nfc * d2 <= 65,536 trace unknowns; larger meshes return HDG_ERR_ARG.
 *   The first call on a device looks up the array's address (with that device current);
 *   make that first call before any stream capture.
 *   All calls share the array and leave their contents in it; the call clears what must
 *   start at zero.  Calls whose GPU work overlaps (other streams or host threads) race.
 * Arguments, outputs and errors as for hdg_solve_trace (x0, uhat device f64 [nfc][d2]; the
 * Dirichlet entries of x0 are ignored; one restarted pass when the recursive residual has
 * converged but the true one has not).  It is the symmetric (CG) solve: a mesh with a
 * convection field returns HDG_ERR_UNSUPPORTED.                                          */
int hdg_solve_trace_noalloc(hdg_mesh* mesh, double rtol, int maxit, const double* x0,
                            double* uhat, int* iters, double* relres);

/* y = H x on the free faces (0 on Dirichlet faces), the trace operator of eq. 6.5 applied
 * matrix-free; x, y device f64 [nfc][d2].                                                 */
int hdg_trace_apply(hdg_mesh* mesh, const double* x, double* y);

/* ------------------------------------------------------------------ learned initial guess
 * (not in the paper).  A continuous piecewise-linear coarse field with values c [nc] at
 * coarse nodes is given through per-vertex interpolation: the value at mesh vertex v is
 * sum_{j<4} weights[4v+j] c[nodes[4v+j]] (nodes < 0 are skipped); nodes int32 and weights
 * f64 [nver][4], device.  On meshes nested in the coarse mesh the field is linear on each
 * element, so its trace on a face is exactly u_hat_e = T [V(w1) V(w2) V(w3)] with
 * T = (varpi . D)^T Xi (eq. 6.3).
 * hdg_prolong:  uhat [nfc][d2] = Pi c (0 on Dirichlet faces).
 * hdg_restrict: c [nc] = Pi^T y (adjoint of hdg_prolong over the free faces).
 * hdg_coarse_solve: the coarse Galerkin problem (Pi^T H Pi) c = Pi^T b by matrix-free CG in
 *   FP64 to rtol (relative to Pi^T b); after hdg_assemble_condense and the boundary data.
 *   It allocates temporary device buffers.                                                */
int hdg_prolong(hdg_mesh* mesh, const int32_t* nodes, const double* weights, const double* coarse,
                double* uhat);
int hdg_restrict(hdg_mesh* mesh, const int32_t* nodes, const double* weights, int64_t nc,
                 const double* y, double* coarse);
int hdg_coarse_solve(hdg_mesh* mesh, const int32_t* nodes, const double* weights, int64_t nc,
                     double* c, double rtol, int maxit, int* iters, double* relres);
/* hdg_fourier_field: sampled coefficient fields for training and evaluating the network.
 * out[i] = g(x_i), or exp(g(x_i)) if exponentiate, for the random Fourier field
 *   g(x) = sigma M^-1/2 sum_m (xi_m cos(omega_m . x) + eta_m sin(omega_m . x)),
 * omega [M][3], amps [2M] = (xi_1..xi_M, eta_1..eta_M); X, Y, Z, out [n]; all device, FP64.
 * 1 <= M <= 1024.  (Input generation for the learned guess; no counterpart in the paper.)  */
int hdg_fourier_field(int64_t n, const double* X, const double* Y, const double* Z, int M,
                      const double* omega, const double* amps, double sigma, int exponentiate,
                      double* out, void* stream);
/* hdg_coarse_guess: x0 [nfc][d2] = alpha Pi c with alpha = (w.b)/(w.Hw), w = Pi c (the
 * energy-optimal multiple; a one-vector coarse correction).  alpha returned on the host.  */
int hdg_coarse_guess(hdg_mesh* mesh, const int32_t* nodes, const double* weights,
                     const double* coarse, double* x0, double* alpha);

/* Kernels of the small network that maps random-field parameters to coarse solutions
 * (FP32, device pointers, enqueued on `stream`):
 * hdg_nn_gemm: C[M][N] = act(sum_k A(m,k) B(k,n) + beta C + bias[n]) with
 *   A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C row stride ldc, bias [N] or
 *   NULL, act 0 (identity) or 1 (tanh).
 * hdg_nn_tanh_bwd: dY[i] *= 1 - Y[i]^2.   hdg_nn_colsum: db[n] = sum_m dZ[m][n].
 * hdg_nn_mse: grad = 2 (pred - target) / n; loss_partial [64] sums to mean((pred - target)^2).
 * hdg_nn_adam: one Adam step (Kingma and Ba 2015) at step number `step` >= 1.           */
int hdg_nn_gemm(int M, int N, int K, const float* A, int sam, int sak, const float* B, int sbk,
                int sbn, float* C, int ldc, float beta, const float* bias, int act, void* stream);
int hdg_nn_tanh_bwd(int64_t n, const float* Y, float* dY, void* stream);
/* hdg_nn_to_f64: y[i] = (double) x[i] (network output -> coarse coefficients).
 * hdg_nn_to_f32: y[i] = (float) x[i] (sampled field -> network input).                    */
int hdg_nn_to_f64(int64_t n, const float* x, double* y, void* stream);
int hdg_nn_to_f32(int64_t n, const double* x, float* y, void* stream);
int hdg_nn_colsum(int M, int N, const float* dZ, float* db, void* stream);
int hdg_nn_mse(int64_t n, const float* pred, const float* target, float* grad,
               float* loss_partial, void* stream);
int hdg_nn_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1,
                float b2, float eps, int step, void* stream);
/* Normalisation of the training targets T [M][N] (device f64, row-major):
 * hdg_nn_colstats: mean[j] = (1/M) sum_i T[i][j], scale[j] = the population standard deviation
 *   of column j, or 1 where it is 0 (device f64 [N] outputs);
 * hdg_nn_standardize: out[i][j] = (T[i][j] - mean[j]) / scale[j] (device f32 [M][N]);
 * hdg_nn_fold_affine: the last layer y = W x + b (W [Nout][Nin], b [Nout], device f32) trained on
 *   standardised targets becomes W <- diag(scale) W, b <- scale o b + mean, so that it returns
 *   the targets themselves.                                                                 */
int hdg_nn_colstats(int64_t M, int N, const double* T, double* mean, double* scale, void* stream);
int hdg_nn_standardize(int64_t M, int N, const double* T, const double* mean, const double* scale, float* out,
                       void* stream);
int hdg_nn_fold_affine(int Nout, int Nin, float* W, float* b, const double* mean, const double* scale,
                       void* stream);

/* ------------------------------------------------------------------ two-level preconditioner
 * (not in the paper, which solves eq. 6.5 directly).  With a coarse space set, the PCG of
 * hdg_solve_trace (both precisions; with convection, right preconditioning of BiCGStab) is preconditioned
 * by M^-1 r = B^-1 r + Pi V(Pi^T r): B the block-Jacobi part, Pi the trace (eq. 6.3 face
 * coefficients) of a continuous piecewise-linear field, V one symmetric V-cycle (one l1-Jacobi
 * sweep before and after each coarse correction, FP32) for A_0 = Pi^T H Pi over nested levels
 * A_{l+1} = P_l^T A_l P_l, exact dense solve on the coarsest level.  The Galerkin matrices are
 * rebuilt on the device after every hdg_assemble_condense (at the next solve).
 * hdg_set_coarse_space: 2 <= nlev <= 17 levels with sizes[l] nodes (sizes[nlev-1] <= 128); host
 *   arrays nodes int32 / weights f64 [R][4], R = nver + sizes[0] + ... + sizes[nlev-2]: first,
 *   per mesh vertex, the level-0 nodes and weights giving its value; then, per node of level
 *   l < nlev-1, the level-(l+1) nodes and weights interpolating it.  Node -1 = unused entry.
 *   Copied; nlev = 0 removes the coarse space.  Every element may touch at most 8 level-0
 *   nodes (HDG_ERR_UNSUPPORTED).  Invalid sizes or nodes: HDG_ERR_ARG.
 * hdg_coarse_precond_apply: z = M^-1 r for device f64 [nfc][d2] vectors starting on 16-byte
 *   boundaries (HDG_ERR_ARG otherwise; Dirichlet entries of r ignored; tests and inspection). */
int hdg_set_coarse_space(hdg_mesh* mesh, int nlev, const int64_t* sizes, const int32_t* nodes,
                         const double* weights);
int hdg_coarse_precond_apply(hdg_mesh* mesh, const double* r, double* z);

/* hdg_autotune: (1) pick the persistent grids of the trace-solve kernels (4 to 32 blocks per
 * SM) and the form of the operator product (one face-major pass over the faces' rows of C^K,
 * or an element pass over contiguous C^K blocks followed by a per-face sum of the owners'
 * contributions), one choice for the FP64 and one for the FP32 iterations, by timing one
 * block-Jacobi PCG iteration (operator, update, direction) of the assembled system in each
 * precision (the environment variable HDG_MATVEC=face|element, read at mesh creation, fixes
 * the form);
 * (2) pick the launch shape of the double-float assembly (threads per element and resident
 * elements per SM: two shapes at k = 1, three at k = 2..4, and for reaction-diffusion at
 * k = 4 two more of a kernel that holds W_* = L^-1 C_*^T one direction at a time, so that
 * three elements stay resident per SM) by timing it.  The choices are kept by the
 * mesh; the system of the caller's last hdg_assemble_condense is restored.  out (nullable,
 * host) receives the choices and the best times.  Requires hdg_assemble_condense
 * (HDG_ERR_STATE) and the boundary data.  Not in the paper.                                */
typedef struct hdg_tuning {
  int face_blocks;    /* FP64 persistent grid (blocks)                  */
  int face_blocks32;  /* FP32 persistent grid (blocks)                  */
  int k1_threads;     /* threads per element of the double-float K1     */
  double iter_ms;     /* one FP64 block-Jacobi iteration at the choice  */
  double iter32_ms;   /* one FP32 iteration at the choice               */
  double k1_ms;       /* one double-float assembly at the choice        */
  int matvec_em64;    /* FP64 solve loops: 1 = element pass + face sum,  */
  int matvec_em32;    /*   0 = one face-major pass; the same for FP32    */
  int k1_streamed;    /* 1: the chosen K1 shape streams W_* (k = 4)      */
} hdg_tuning;
int hdg_autotune(hdg_mesh* mesh, hdg_tuning* out);

/* Relative tolerance of each FP32 inner solve of the HDG_MIXED_FP32 trace solve (default
 * 1e-4): every outer FP64 refinement step asks the inner PCG (BiCGStab with convection) for
 * this residual reduction, or only for half the remaining distance to rtol ||b|| when that is
 * less (the last step stops as soon as it suffices).                                       */
int hdg_set_inner_tolerance(hdg_mesh* mesh, double rtol);

/* Residual check (tests): r = b - H x over the free dofs, device f64 [nfc][d2]; returns
 * ||r||_2 and ||b||_2 through the host pointers.                                          */
int hdg_trace_residual(hdg_mesh* mesh, const double* x, double* r, double* rnorm, double* bnorm);

/* Local recovery (eq. 5.3): q [nelt][3][n], u [nelt][n] device f64 outputs from the trace
 * uhat [nfc][d2] (device f64); in double-float arithmetic after an HDG_DF32 assembly (a
 * record copy that never lands, which only a hardware fault could cause, leaves NaN and is
 * reported by the next assembly as HDG_ERR_CUDA).                                         */
int hdg_recover(hdg_mesh* mesh, const double* uhat, double* q, double* u);

/* The same recovery into host arrays q [nelt][3][n], u [nelt][n] (page-locked for overlap):
 * the elements in `chunks` ranges, each range's device -> host copy running while the next
 * range is recovered.  uhat device f64 [nfc][d2].  Synchronises.                          */
int hdg_recover_host(hdg_mesh* mesh, const double* uhat, double* q, double* u, int chunks);

/* Superconvergent postprocess (eq. 9.11): ustar [nelt][n1] device f64 (coefficients in the
 * degree-(k+1) Dubiner basis) from q, u of hdg_recover; kappa as set by
 * hdg_set_coefficients; in double-float arithmetic after an HDG_DF32 assembly.           */
int hdg_postprocess(hdg_mesh* mesh, const double* q, const double* u, double* ustar);

/* ------------------------------------------------------------------ projections and error norms
 * Diagnostics of Section 9 ("Error functions", "HDG projection") and eq. 10.1-10.2.  FP64.
 *
 * hdg_projection: the HDG projection of eq. 9.13, (Pi q, Pi u) in P_k(K)^3 x P_k(K) with
 *   (Pi q, r)_K = (q, r)_K for r in P_{k-1}(K)^3, (Pi u, w)_K = (u, w)_K for w in P_{k-1}(K),
 *   <Pi q.nu + tau Pi u, v>_dK = <q.nu + tau u, v>_dK for v in R_k(dK), tau as set by
 *   hdg_set_coefficients (1 when none was given).  Inputs (device f64): q_vol [3][nelt][nq]
 *   and u_vol [nelt][nq] at the volume nodes (hdg_quadrature_nodes); q_face [3][nelt][4][nf]
 *   and u_face [nelt][4][nf] at the element-local face nodes (hdg_element_face_nodes).
 *   Outputs (device f64): Pq [nelt][3][n], Pu [nelt][n] (Dubiner coefficients, as hdg_recover).
 *   Synchronises the mesh's stream.  HDG_ERR_LOCAL_SINGULAR if an element's m x m face
 *   system has a zero pivot (its outputs are NaN); HDG_ERR_ARG for NULL pointers.
 * hdg_face_projection: the L2 projection onto P_k(e) of eq. 9.12 on every face, from the
 *   values vals [nfc][nf] at the face nodes (hdg_quadrature_nodes); Pu [nfc][d2] device f64.
 * hdg_volume_norm2: out[0] = sum_K |K| sum_q omega_q (vals - sum_j coef_j P_j)^2 and
 *   out[1] = sum_K |K| sum_q omega_q vals^2 on the volume rule (host double[2]); coef
 *   [nelt][dim] in the degree-`degree` basis (degree k: dim = n, as u_h; degree k + 1:
 *   dim = n1, as u_h*) or NULL (zero), vals [nelt][nq] or NULL (zero).  Synchronises.
 * hdg_face_norm2: out[0] = ||vals - sum_a coef_a D_a||_h^2 and out[1] = ||vals||_h^2 with
 *   ||v||_h^2 = sum_e |e| ||v||_e^2 (eq. 10.2) on the face rule; coef [nfc][d2] or NULL,
 *   vals [nfc][nf] or NULL.  Synchronises.
 * The ratios of eq. 10.1-10.2 follow: e_h^u = sqrt(out[0] / out[1]) with coef = u_h and vals =
 * u; eps_h^u with coef = Pi u - u_h and vals = u for the reference; eps_h^uhat with the face
 * norms of P u - uhat_h and of u.  Sums are deterministic (fixed two-level order).        */
int hdg_projection(hdg_mesh* mesh, const double* q_vol, const double* u_vol, const double* q_face,
                   const double* u_face, double* Pq, double* Pu);
int hdg_face_projection(hdg_mesh* mesh, const double* vals, double* Pu);
int hdg_volume_norm2(hdg_mesh* mesh, int degree, const double* coef, const double* vals, double* out);
int hdg_face_norm2(hdg_mesh* mesh, const double* coef, const double* vals, double* out);

/* ------------------------------------------------------------------ dense contraction on tensor cores
 * The volume masses of eq. 3.55 as one dense contraction for all elements,
 *   out[e][p] = sum_q |K_e| omega_q g[e][q] P_i(p_hat_q) P_j(p_hat_q),  p = (i <= j) in the
 *   row-major order of the upper triangle (n(n+1)/2 pairs),
 * i.e. the GEMM [nelt x nq] . [nq x n(n+1)/2].  A measurement of that contraction on its own,
 * not a step of the solver: hdg_assemble_condense forms the masses by sum factorisation and
 * keeps FP64-level accuracy, which BF16 operands cannot.
 *   mode 0: 5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation);
 *   mode 1: CUDA cores, FP32 arithmetic on the same BF16-rounded operands (the reference of
 *           mode 0: the two differ only by the order of the FP32 additions);
 *   mode 2: CUDA cores, FP32 operands and arithmetic.
 *   g: device f64 [nelt][nq] (the coefficient at the volume nodes, e.g. 1/kappa);
 *   out: device f32 [nelt][n(n+1)/2].
 * Synchronises the mesh's stream in mode 0 and returns HDG_ERR_CUDA if a tensor-core wait ran
 * out (bounded waits; the kernel frees its tensor memory in that case).  k >= 1.          */
int hdg_mass_contraction(hdg_mesh* mesh, const double* g, int mode, float* out);

/* The masses of the HDG_MIXED_BF16 assembly for the current coefficients, on their own (tests,
 * measurement): out device f32 [nelt][*stride] = [M_{kappa^-1} pairs | M_c pairs | f^K | pad],
 * pairs (i <= j) in row-major order (i = 0: j = 0..n-1, then i = 1, ...), so the f^K entries
 * follow the 2 n(n+1)/2 pair entries; *stride (host, nullable) = n(n+1) + n rounded up to a
 * multiple of 4.  With out NULL only *stride is set.  One tensor-core contraction over all
 * elements (each FP64 operand split into three BF16 parts, six products, FP32 accumulation).
 * HDG_ERR_UNSUPPORTED for k = 0 or the symmetric rule, HDG_ERR_COEFF for kappa <= 0, c < 0 or
 * non-finite data, HDG_ERR_CUDA if an MMA does not complete within the bounded wait.       */
int hdg_mixed_masses(hdg_mesh* mesh, float* out, int* stride);

/* ------------------------------------------------------------------ batched problems
 * Many independent problems of mixed degree solved together.  Problems of equal degree are
 * merged into one disjoint-union mesh (a "group"), so each phase is one launch per group, and
 * the whole batch (assembly + condensation, boundary data, PCG run on the device until
 * convergence, recovery) is one CUDA graph launch with one branch per group.
 * hdg_batch_create: per problem p, host arrays as for hdg_mesh_create (coords[p] [nver[p]][3],
 *   elems[p] [nelt[p]][4], dir[p] [ndir[p]][3], neu[p] [nneu[p]][3]) and degree k[p] in 1..4.
 * hdg_batch_group: the union mesh of group g (owned by the batch: set its coefficients and
 *   boundary data with hdg_set_coefficients / hdg_set_boundary_data, query its nodes with
 *   hdg_quadrature_nodes), its degree, its problems (prob_ids [np]) and their element and
 *   face ranges in the union (elem_off, face_off [np+1]); any output pointer may be NULL.
 * hdg_batch_run: precision HDG_FP64 or HDG_DF32 (assembly arithmetic), PCG iterated until
 *   ||r|| <= rtol min_p ||b_p|| (so every problem meets rtol).  relres [nprob] host:
 *   per-problem ||b_p - H_p u_p|| / ||b_p||; iters [ngroups] host (inner iterations for the
 *   mixed solve).  HDG_ERR_NOT_CONVERGED if some problem misses rtol within maxit.  A group
 *   mesh with a coarse space (hdg_set_coarse_space) uses the two-level preconditioner.
 * hdg_batch_set_solve_precision: HDG_FP64 (default) or HDG_MIXED_FP32: FP64 residuals and
 *   updates around FP32 inner PCG solves (each to the group mesh's inner tolerance), both
 *   loops driven on the device inside the batch graph (nested conditional WHILE nodes).
 * hdg_batch_solution: device pointers (owned by the batch) to the group's u_hat [nfc][d2],
 *   q [nelt][3][n], u [nelt][n] in union numbering.                                        */
typedef struct hdg_batch hdg_batch;
int hdg_batch_create(int nprob, const double* const* coords, const int64_t* nver,
                     const int32_t* const* elems, const int64_t* nelt,
                     const int32_t* const* dir, const int64_t* ndir,
                     const int32_t* const* neu, const int64_t* nneu, const int* k,
                     void* stream, hdg_batch** out);
int hdg_batch_num_groups(const hdg_batch* batch, int* ngroups);
int hdg_batch_group(const hdg_batch* batch, int g, hdg_mesh** mesh, int* k, int* np,
                    int32_t* prob_ids, int64_t* elem_off, int64_t* face_off);
int hdg_batch_run(hdg_batch* batch, int precision, double rtol, int maxit, double* relres,
                  int* iters);
int hdg_batch_set_solve_precision(hdg_batch* batch, int precision);
int hdg_batch_solution(const hdg_batch* batch, int g, double** uhat, double** q, double** u);
int hdg_batch_destroy(hdg_batch* batch);

/* Copy the message of the calling thread's last error into buf (NUL-terminated). */
int hdg_last_error(char* buf, size_t len);

/* Number of kernel launches this handle has enqueued so far (instrumentation). */
int64_t hdg_launch_count(const hdg_mesh* mesh);

/* Host-only helpers (no GPU needed), used to check the library's host logic.
 * hdg_host_table: copy the reference table `name` of degree k into out (host f64, at least
 *   *size entries; out may be NULL to query *size; "<name>:sym" gives the table of the
 *   symmetric volume rule of hdg_set_volume_rule).  Names and layouts (row-major):
 *   vol_pts [nq][3], vol_w [nq], P [nq][n], Pd [3][nq][n], Chat [3][n][n] (eq. 3.5-3.7),
 *   face_pts [nf][2], face_w [nf], Pl [4][nf][n], D [nf][d2], Dmu [6][nf][d2] (eq. 4.4, 4.7),
 *   S [4][n][n] (eq. 4.5 pieces), E [4][6][d2][n] (eq. 4.10 pieces),
 *   P1 [nq][n1], G1 [3][nq][n1], Shat1 [6][n1][n1] (degree k+1, eq. 9.11); the sum-
 *   factorisation tables of the volume masses: sfAA [np1][k+2], sfBB [np2][k+2],
 *   sfCC [n(n+1)/2][k+2] (pair products of the collapsed-coordinate factors of the basis),
 *   sfp2to1 [np2] and sfp3to2 [n(n+1)/2] (pair maps, as doubles).
 * hdg_host_expand_mesh: the expanded mesh of Section 2 on the host.  faces needs room for
 *   4 nelt rows of 4 (nfc <= 4 nelt), facebyele and perm [nelt][4]; *nfc receives the count. */
int hdg_host_table(int k, const char* name, double* out, int64_t capacity, int64_t* size);
int hdg_host_expand_mesh(const double* coords, int64_t nver, const int32_t* elems, int64_t nelt,
                         const int32_t* dir, int64_t ndir, const int32_t* neu, int64_t nneu,
                         int64_t* nfc, int32_t* faces, int32_t* facebyele, int32_t* perm);

#ifdef __cplusplus
}
#endif
#endif /* HDG_H */
