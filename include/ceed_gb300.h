/*
 * ceed_gb300.h -- C ABI of the GB300 (sm_103a) matrix-free hexahedral operator library.
 *
 * The library computes the action y = A x of the high-order finite-element mass and
 * diffusion operators on hexahedral meshes without assembling A (paper Section 2:
 * A_L = block-diag(A^e), A^e = D^T G^e D, applied element by element with sum-factorized
 * tensor contractions), and a preconditioned conjugate-gradient solver on top of it
 * (Section 1: CG with a cheap preconditioner on the matrix-free operator).
 *
 * Conventions for every entry point:
 *  - Every call returns an int status (ceed_status); none aborts or throws across the ABI.
 *    On failure ceed_last_error() returns a message (thread-local).
 *  - Vectors, quadrature data, coefficient fields and workspaces are CALLER-OWNED device
 *    memory (e.g. torch tensors).  The mesh handle owns only the tables it builds at setup
 *    (colour-sorted restriction, element permutation, a copy of the vertices, 1D bases).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Apply
 *    calls are asynchronous on it and OVERWRITE y (they do not accumulate into it).
 *  - Numbering: element nodes n = a + P (b + P c) (a along r fastest, P = p + 1); quadrature
 *    points q = i + Q (j + Q k).  Per-element, per-point arrays passed by the caller
 *    (coefficients, dL/dk) are [n_elem][Q^3] in the caller's element order.
 *  - L-vectors hold ncomp * nrhs interleaved columns: entry (dof, comp, rhs) lives at
 *    (dof * ncomp + comp) * nrhs + rhs.  All L-vectors are FP64.
 */
#ifndef CEED_GB300_H
#define CEED_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ceed_mesh_s *ceed_mesh_t;

typedef enum {
  CEED_OK = 0,
  CEED_ERR_INVALID = 1,        /* bad argument (size, pointer, out-of-range index, unsupported p) */
  CEED_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  CEED_ERR_OOM = 3,            /* device or host allocation failed */
  CEED_ERR_NOT_CONVERGED = 4,  /* solver hit its iteration cap (report still filled) */
  CEED_ERR_UNSUPPORTED = 5,    /* valid request this build does not implement */
  CEED_ERR_BAD_GEOMETRY = 6,   /* det J <= 0 at some quadrature point */
  CEED_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
  CEED_ERR_NONFINITE = 8       /* NaN/Inf met in a solver reduction */
} ceed_status;

/* Precision of stored quadrature data; it also selects the operator arithmetic:
 * F64 -> FP64 contractions; F32/BF16/F16 -> FP32 contractions (FP64 L-vectors in and out).
 * F32_GEO (diffusion only) -> FP32 contractions with the geometric factors recomputed from the
 * trilinear element map at every application: the quadrature data holds only the map's 8
 * coefficient vectors per element and w k per point (FP32), about 1/6 of the F32 bytes.
 * F64_DF (mass and diffusion, either rule) -> an FP64-accurate operator computed on the FP32 pipe:
 * values and quadrature data carried as double-float pairs (hi + lo, about 48 bits) and every
 * contraction summed with a compensated dot product; agrees with the FP64 operator to ~1e-14
 * relative on well-conditioned inputs (FP64 L-vectors in and out, qdata 8 bytes per value).  Each
 * word must stay in the FP32 normal range: with the quadrature data of unit-cube meshes the 1e-12
 * agreement holds for inputs of magnitude 1e-20 .. 1e30 (tested; at 1e-30 it fails); beyond that
 * range the low words underflow (accuracy falls towards FP32) or the high words overflow (Inf). */
typedef enum { CEED_F64 = 0, CEED_F32 = 1, CEED_BF16 = 2, CEED_F16 = 3, CEED_F32_GEO = 4, CEED_F64_DF = 5 } ceed_prec;

/* Quadrature: GLL = collocated on the p+1 Gauss-Lobatto nodes (BP5 style, Q = p+1);
 * GAUSS = Q Gauss-Legendre points per direction (BP1/BP3 style, default Q = p+2). */
typedef enum { CEED_QRULE_GLL = 0, CEED_QRULE_GAUSS = 1 } ceed_qrule;

typedef enum { CEED_OP_MASS = 0, CEED_OP_DIFFUSION = 1 } ceed_op;

/* Coefficient (rho for mass, k for diffusion):
 *  ONE       1 everywhere                       coeff ignored (may be NULL)
 *  CONST     coeff[0] (host pointer)            a positive constant
 *  SINE      1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z) at the physical quadrature points
 *  PER_QPT   device array [n_elem][Q^3], caller's element order                        */
typedef enum { CEED_COEFF_ONE = 0, CEED_COEFF_CONST = 1, CEED_COEFF_SINE = 2, CEED_COEFF_PER_QPT = 3 } ceed_coeff;

/* Apply flags. */
#define CEED_APPLY_DIRICHLET 1u  /* rows/columns of Dirichlet nodes replaced by the identity */
#define CEED_APPLY_F64_DF 2u     /* per-point-coefficient operator and adjoint: FP64 accuracy on the FP32
                                    pipe (double-float arithmetic; needs the stored geometry) */

typedef struct {
  int64_t n_elem;            /* E >= 1 */
  int64_t n_ldof;            /* nodes in the L-vector, < 2^29 */
  int32_t p;                 /* polynomial order, 1..8 */
  int32_t q_rule;            /* ceed_qrule */
  int32_t n_qpts_1d;         /* Q; 0 selects the default (p+1 for GLL, p+2 for GAUSS); GAUSS needs Q = p+2 */
  int32_t ncomp;             /* components per node (>= 1), sharing one operator (A (x) I) */
  const int32_t *elem_dofs;  /* device [E][(p+1)^3], 0 <= dof < n_ldof, every dof referenced */
  const double *vertices;    /* device [E][8][3], trilinear element map, vertex v = vx + 2 vy + 4 vz */
  const uint8_t *dirichlet;  /* device [n_ldof] (nonzero = Dirichlet node) or NULL */
  const double *coords;      /* device [n_ldof][3] physical node positions of a curved (isoparametric,
                              * degree-p) geometry, or NULL for the trilinear map of `vertices`.  With
                              * coords, quadrature data and right-hand sides use x(xi) = sum_n phi_n(xi)
                              * x_n; F32_GEO data and the adjoint's recomputed geometry (both built on
                              * the trilinear map) are refused with UNSUPPORTED. */
} ceed_mesh_desc;

/* Build a mesh handle (paper Section 2: the element restriction and 1D bases of the
 * factored operator).  Copies elem_dofs/vertices/dirichlet to the host, validates them,
 * colours the elements greedily so that no two elements of one colour share a node, and
 * uploads a colour-sorted restriction with first-writer and Dirichlet flags (this is what
 * makes the scatter-add atomic-free and deterministic).  The caller's arrays may be freed
 * afterwards.  Synchronizes `stream`.  Errors: INVALID (sizes, p, out-of-range or
 * unreferenced dof), UNSUPPORTED (more than 64 colours), OOM, CUDA. */
int ceed_setup_mesh(const ceed_mesh_desc *desc, ceed_mesh_t *out, void *stream);

/* Physical positions of every node, device [n_ldof][3]: the handle's curved-geometry copy if it
 * has one, else the trilinear map of each element at its GLL nodes (the isoparametric form of the
 * trilinear geometry; a caller can move these points and set up a curved mesh from them).
 * Asynchronous on `stream`.  Errors: INVALID. */
int ceed_mesh_node_coords(ceed_mesh_t mesh, double *coords, void *stream);

/* Release a handle and its device tables (NULL is a no-op).  Synchronizes the device. */
int ceed_destroy_mesh(ceed_mesh_t mesh);

/* Mesh facts: number of colours, points per direction Q, nodes per direction P. */
int ceed_mesh_info(ceed_mesh_t mesh, int32_t *n_colors, int32_t *Q, int32_t *P);

/* Bricks found at setup (Section 2's gather and scatter grouped over neighbouring elements): the
 * number of 2 x 2 x 1 element groups of a structured lattice -- node numbering x fastest, every
 * element's nodes at base + a + b sy + c sz with common strides, even element counts per direction
 * -- or 0 when the mesh is not such a lattice.  On a brick mesh the FP32-pipe operators (F32, BF16,
 * F16, F32_GEO) with one column may run the brick kernel (apply variant stages 2 and 3), which reads
 * every node of a brick once instead of once per element that contains it. */
int ceed_mesh_bricks(ceed_mesh_t mesh, int64_t *n_bricks);

/* Bytes of quadrature data for (op, prec): mass 1 value per point, diffusion 6 (the
 * symmetric G_rr, G_rs, G_rt, G_ss, G_st, G_tt of Section 2).  Layout is internal:
 * [colour-sorted element][component][Q^3]. */
size_t ceed_qdata_bytes(ceed_mesh_t mesh, int op, int prec);

/* Compute quadrature data (Section 2: the six diagonal matrices of the symmetric tensor
 * G^e; mass: w |det J| rho).  Diffusion: G = w k adj(J) adj(J)^T / det J.  Writes
 * ceed_qdata_bytes(mesh, op, prec) bytes to `qdata` (device).  Synchronizes `stream` to
 * report BAD_GEOMETRY if det J <= 0 anywhere. */
int ceed_build_qdata(ceed_mesh_t mesh, int op, int coeff_kind, const double *coeff, int prec,
                     void *qdata, void *stream);

/* y = M x: matrix-free mass action (BP1).  x, y device FP64 [n_ldof * ncomp * nrhs],
 * x and y must not overlap.  `prec` is the precision qdata was built in. */
int ceed_apply_mass(ceed_mesh_t mesh, const void *qdata, int prec, const double *x, double *y,
                    int nrhs, unsigned flags, void *stream);

/* y = A x: matrix-free diffusion action (BP3/BP5), Section 2's A_L u_L.  One fused kernel
 * per colour: gather (L->E), 1D contractions to quadrature points, pointwise G^e, transposed
 * contractions, scatter-add (E->L) without atomics.  Same argument rules as ceed_apply_mass. */
int ceed_apply_diffusion(ceed_mesh_t mesh, const void *qdata, int prec, const double *x, double *y,
                         int nrhs, unsigned flags, void *stream);

/* Host-buffer form of the two actions (Section 2's A_L u_L, as ceed_apply_mass / ceed_apply_diffusion),
 * for callers whose vectors live in host memory: copies
 * x_host into the caller's device buffer x_dev, applies the operator `op` (CEED_OP_MASS or
 * CEED_OP_DIFFUSION; qdata, prec, nrhs, flags as for ceed_apply_mass / ceed_apply_diffusion) into
 * y_dev, and copies y_dev into y_host, all on `stream`, and returns once y_host holds the result
 * (synchronizes `stream`).  x_host, y_host: host FP64 [n_ldof * ncomp * nrhs]; page-locked memory
 * copies at full link bandwidth, pageable memory goes through the driver's staging.  x_dev, y_dev:
 * device FP64 of the same size, caller-owned, not overlapping.  Errors: INVALID, CUDA. */
int ceed_apply_host(ceed_mesh_t mesh, int op, const void *qdata, int prec, const double *x_host, double *y_host,
                    double *x_dev, double *y_dev, int nrhs, unsigned flags, void *stream);

/* Autotuner (the batched-apply design calls for tile shape and elements per block chosen by
 * measurement): runs every variant of the fused apply kernel -- elements per thread block
 * (1, 2, 4, ... up to 256 threads and 32 elements) x quadrature-data staging (TMA bulk copy into shared memory,
 * or direct loads), and the brick kernel with and without staging where the mesh and precision
 * allow it (ceed_set_apply_variant) -- on the caller's qdata, x and y (y is overwritten), times each with CUDA
 * events on `stream`, and keeps the fastest in the handle for (op, prec); later applies use it.
 * Returns the choice and its time per application.  Synchronizes `stream`. */
int ceed_autotune_apply(ceed_mesh_t mesh, int op, const void *qdata, int prec, const double *x, double *y,
                        int nrhs, int32_t *best_ne, int32_t *best_stage, float *best_ms, void *stream);

/* Fix the apply variant for (op, prec) by hand: ne elements per thread block (0 restores the
 * default), stage = 1 for TMA staging of quadrature data, 0 for direct loads; stage = 2 (direct
 * loads) or 3 (staging) selects the brick kernel, one 2 x 2 x 1 element group per thread block (ne
 * is then ignored), for the FP32-pipe precisions on meshes with bricks (ceed_mesh_bricks).  INVALID
 * if ne exceeds min(32, 256 / Q^2), or for a brick stage the mesh or precision cannot use.  The
 * element variants (stages 0, 1) give bitwise-identical results; the brick variants add the
 * contributions to a shared node in another order (the brick's elements first), so they agree
 * with them to FP32 rounding, deterministically.  A brick choice applies to single-column applies;
 * several columns run the default element variant. */
int ceed_set_apply_variant(ceed_mesh_t mesh, int op, int prec, int ne, int stage);

/* Jacobi diagonal of the operator (the cheap preconditioner for CG, Section 1), FP64
 * [n_ldof * ncomp] (one value per node and component); with CEED_APPLY_DIRICHLET the
 * Dirichlet entries are 1. */
int ceed_jacobi_diagonal(ceed_mesh_t mesh, int op, const void *qdata, int prec, double *diag,
                         unsigned flags, void *stream);

/* Right-hand side b_i = sum_e sum_q w |det J| f(x_q) phi_i(x_q) for the manufactured solution
 * u* = sin(pi x) sin(pi y) sin(pi z), f = -div(k grad u*), k = coeff_kind (ONE or SINE),
 * integrated with the mesh's quadrature.  Zero on Dirichlet nodes with CEED_APPLY_DIRICHLET.
 * b: device FP64 [n_ldof] (ncomp must be 1). */
int ceed_manufactured_rhs(ceed_mesh_t mesh, int coeff_kind, double *b, unsigned flags, void *stream);

/* ---------------------------------------------------------------- batched apply */

/* Several independent meshes -- polynomial orders may differ -- applied by ONE persistent kernel
 * launch (multi-right-hand-side batching and mixed order in one launch).  The launch is sized to the
 * thread blocks that are co-resident on the GPU; each block loops over the colours and over its share
 * of every mesh's elements of that colour, with a bounded grid-wide barrier between colours (the
 * atomic-free scatter needs colours in sequence).  The launch is captured once into a CUDA graph and
 * replayed by ceed_batch_apply.  Buffers are fixed at creation: qdata[k] (built for meshes[k] in
 * `prec`), x[k], y[k] (FP64, [n_ldof * ncomp * nrhs] of mesh k).  All meshes must use the same
 * quadrature rule kind (GLL or Gauss).  Supported: F64 and F64_DF (the FP64-accurate double-float
 * operator) mass/diffusion, F32 diffusion.  The batch must
 * not run concurrently with other kernels on the device (the persistent grid assumes it has the GPU);
 * if a barrier wait times out, ceed_batch_status returns CEED_ERR_TIMEOUT. */
typedef struct ceed_batch_s *ceed_batch_t;
int ceed_batch_create(int n, const ceed_mesh_t *meshes, const void *const *qdata, int prec, int op,
                      const double *const *x, double *const *y, int nrhs, ceed_batch_t *out);
/* y[k] = A_k x[k] for every mesh of the batch, one graph launch on `stream`. */
int ceed_batch_apply(ceed_batch_t batch, void *stream);
/* Autotuner: times threads per block (128, 192, 256; elements per block = threads / Q^2 for each
 * mesh) x quadrature-data staging on the batch's own buffers, keeps the fastest and re-captures the
 * graph.  Synchronizes `stream`. */
int ceed_batch_autotune(ceed_batch_t batch, float *best_ms, void *stream);
/* Launch shape in use: threads per block, staging, blocks in the persistent grid. */
int ceed_batch_info(ceed_batch_t batch, int32_t *threads, int32_t *stage, uint32_t *grid);
/* Synchronizes `stream`; CEED_ERR_TIMEOUT if a bounded device wait of an earlier launch gave up. */
int ceed_batch_status(ceed_batch_t batch, void *stream);
int ceed_batch_destroy(ceed_batch_t batch);

/* ---------------------------------------------------------------- CG solver */

typedef enum { CEED_CG_FP64 = 0, CEED_CG_MIXED = 1, CEED_CG_MIXED_RELIABLE = 2 } ceed_cg_mode;

typedef struct ceed_pmg_s *ceed_pmg_t;

typedef struct {
  int32_t mode;           /* ceed_cg_mode */
  int32_t max_iter;       /* cap on (inner) iterations in total; 0 -> 10000 */
  int32_t max_outer;      /* MIXED: cap on refinement steps; 0 -> 50 (MIXED_RELIABLE: unused) */
  int32_t check_every;    /* host convergence check period in iterations; 0 -> 10 */
  int32_t fixed_iters;    /* > 0: run exactly this many FP64 iterations (no tolerance stop) */
  int32_t op;             /* ceed_op of the operator (DIFFUSION for the bake-off CG) */
  double tol;             /* stop when ||b - A x||_2 <= tol ||b||_2; 0 -> 1e-10 */
  double inner_tol;       /* MIXED: inner relative reduction; 0 -> 1e-4 */
  const void *qdata_lo;   /* MIXED, MIXED_RELIABLE: quadrature data for the low-precision operator */
  int32_t prec_lo;        /* MIXED, MIXED_RELIABLE: its precision (F32, BF16, F16, F32_GEO or F64_DF) */
  int32_t use_x0;         /* nonzero: x holds the initial guess; else x0 = 0 */
  ceed_pmg_t pmg;         /* FP64 mode: non-NULL -> flexible CG preconditioned by one p-multigrid
                             V-cycle per iteration instead of Jacobi */
  double reliable_delta;  /* MIXED_RELIABLE: replace the recurrence residual by the true FP64 residual
                             each time it has fallen by this factor; 0 -> 0.1, else in (0, 1) */
  int32_t separate_kernels; /* 0: Jacobi-PCG iterations run as one persistent kernel per batch of
                               check_every iterations where the (inner) operator allows it (diffusion,
                               GLL collocated, F64 / F32 / BF16 / F32_GEO / F64_DF); nonzero: one kernel
                               per step (apply, reductions, updates) */
} ceed_cg_opts;

typedef struct {
  int32_t iterations;       /* FP64 CG iterations, or inner iterations summed over refinements */
  int32_t outer_iterations; /* MIXED: refinement steps; MIXED_RELIABLE: FP64 true-residual evaluations */
  double rel_residual;      /* ||b - A x|| / ||b|| with the FP64 operator at exit */
  double seconds;           /* wall time of the solve, measured with CUDA events */
  int32_t fused;            /* 1 if the (inner) PCG iterations ran in the fused persistent kernel */
} ceed_cg_report;

/* Bytes of device workspace ceed_cg_solve needs for these options. */
size_t ceed_cg_workspace_bytes(ceed_mesh_t mesh, const ceed_cg_opts *opts);

/* Solve A x = b with Jacobi-preconditioned CG (Section 1) on the Dirichlet-masked operator.
 * Fused iteration (default where supported): one cooperative persistent kernel runs check_every
 * whole iterations -- the colour-ordered apply q = A p with p.q summed by each node's last writer,
 * alpha, x and r updates with the r.z and r.r sums (z = D^{-1} r is not stored), beta, p update --
 * separated by bounded grid barriers; reductions in a fixed order (results are reproducible run to
 * run, and differ from the separate-kernel path only in rounding order).  A barrier that gives up
 * returns CEED_ERR_TIMEOUT.
 * FP64 mode: all arithmetic FP64.  MIXED mode: iterative refinement, outer residual
 * r = b - A x with the FP64 operator (qdata, prec), inner PCG with the low-precision operator
 * (opts->qdata_lo, FP32 contractions, or the double-float operator of F64_DF) and FP64 vectors,
 * dot products and updates; x += d; each inner pass reduces its residual by inner_tol, or by less
 * when that is all the tolerance still needs.  MIXED_RELIABLE mode: one PCG run with the
 * low-precision operator and FP64 vectors whose recurrence residual is replaced by the true FP64
 * residual b - A x each time it has fallen by reliable_delta (reliable updates, Sleijpen and
 * van der Vorst 1996), keeping the search direction; it stops when the true residual meets tol.
 * b, x: device FP64 [n_ldof] (ncomp = 1).  work: device, ceed_cg_workspace_bytes bytes,
 * 256-byte aligned.  Synchronizes `stream`.  Returns NOT_CONVERGED (report filled) on the cap,
 * NONFINITE on a NaN/Inf reduction. */
int ceed_cg_solve(ceed_mesh_t mesh, const void *qdata, int prec, const double *b, double *x,
                  const ceed_cg_opts *opts, ceed_cg_report *report, void *work, size_t work_bytes,
                  void *stream);

/* ---------------------------------------------------------------- p-multigrid */

/* p-multigrid preconditioner (paper Section 1: p-multigrid as the usual replacement of low-order
 * preconditioners for the matrix-free operator).  Levels are meshes of decreasing order on the SAME
 * elements (meshes[0] finest; all with the same Dirichlet nodes, ncomp = 1, GLL collocated or all
 * Gauss).  Transfers: prolongation evaluates the coarse element polynomial at the fine nodes,
 * restriction is its exact transpose.  Smoother: Chebyshev iteration on D^{-1} A over
 * [lambda_max / smooth_ratio, 1.1 lambda_max] (lambda_max by power iteration at creation), degree
 * smooth_degree before and after the coarse correction.  Coarsest level: Jacobi-PCG to a relative
 * residual coarse_tol (at most coarse_max_iter iterations).  qdata64[l]: FP64 diffusion qdata of
 * level l (Jacobi diagonal, and the smoother unless qdata_lo is given); qdata_lo[l] (may be NULL)
 * with prec_lo selects an FP32-arithmetic smoothing operator.  The handle allocates its level
 * vectors at creation (several n_ldof-sized FP64 vectors per level).  Synchronizes `stream`. */
typedef struct {
  int32_t smooth_degree;    /* 0 -> 4 */
  double smooth_ratio;      /* <= 1 -> 10 */
  int32_t eig_iters;        /* 0 -> 20 */
  double coarse_tol;        /* 0 -> 3e-2 */
  int32_t coarse_max_iter;  /* 0 -> 500 */
  int32_t prec_lo;          /* precision of qdata_lo (F32, BF16, F16, F32_GEO) */
  int32_t smoother;         /* 0: Chebyshev on D^{-1} A (Jacobi); 1: Chebyshev on M A with the overlapping
                               Schwarz smoother M of ceed_schwarz_create (levels must be GLL collocated) */
  int32_t smoother_coeff;   /* smoother 1: coefficient kind for the element means (ONE or SINE) */
} ceed_pmg_opts;

int ceed_pmg_create(int nlevels, const ceed_mesh_t *meshes, const void *const *qdata64, const void *const *qdata_lo,
                    const ceed_pmg_opts *opts, ceed_pmg_t *out, void *stream);
/* z = M r: one V-cycle (r, z device FP64 [n_ldof of level 0]). */
int ceed_pmg_vcycle(ceed_pmg_t pmg, const double *r, double *z, void *stream);
/* Transfers between levels l+1 (coarse) and l (fine): uf = P uc, rc = P^T rf. */
int ceed_pmg_prolong(ceed_pmg_t pmg, int level, const double *uc, double *uf, void *stream);
int ceed_pmg_restrict(ceed_pmg_t pmg, int level, const double *rf, double *rc, void *stream);
/* lambda_max estimate used for level l's smoother: of D^{-1} A (smoother 0) or of M A (smoother 1). */
int ceed_pmg_info(ceed_pmg_t pmg, int level, double *lambda_max);
int ceed_pmg_destroy(ceed_pmg_t pmg);

/* Overlapping Schwarz smoother with fast diagonalization (Section 1's Schwarz/fast-diagonalization
 * preconditioning; the method of Lottes and Fischer, J. Sci. Comput. 24, 2005).  Each element's local
 * problem is its own GLL nodes with Dirichlet conditions one node into each neighbour; its operator
 * is replaced by the separable operator of a box with the element's mean side lengths h_d (mean of the
 * four element edges along each reference axis) and mean coefficient k (over its GLL nodes):
 *   A_e = k (B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x + A_z (x) B_y (x) B_x),  A_d = (2/h_d) A^, B_d = (h_d/2) B^,
 * (A^, B^) the GLL stiffness and mass of three reference elements side by side restricted to the
 * middle one, inverted by fast diagonalization (A^ S = B^ S L, S^T B^ S = I).  The smoother is
 * z = sum_e R_e^T W A_e^{-1} W R_e r, W = diag(multiplicity^{-1/2}) (symmetric), FP32 arithmetic.
 * Requires a GLL collocated mesh with one component.  Coefficient ONE, CONST (host value) or SINE. */
typedef struct ceed_schwarz_s *ceed_schwarz_t;
/* The smoother's 1D fast-diagonalization basis for order p (1..8), in FP64 (the smoother keeps an
 * FP32 copy): S [P][P] with S[a * P + i] eigenvector i at GLL node a, lambda [P], such that
 * A^ S = B^ S diag(lambda) and S^T B^ S = I for the (A^, B^) above; eigenvalues in no particular
 * order.  Host arrays, no GPU work.  Errors: INVALID. */
int ceed_schwarz_fdm_1d(int p, double *S, double *lambda);
int ceed_schwarz_create(ceed_mesh_t mesh, int coeff_kind, const double *coeff, ceed_schwarz_t *out, void *stream);
/* z = M r (device FP64 [n_ldof], no overlap); CEED_APPLY_DIRICHLET: zero on Dirichlet nodes in r and z.
 * Asynchronous; one kernel launch per colour (colour-ordered, deterministic). */
int ceed_schwarz_apply(ceed_schwarz_t sw, const double *r, double *z, unsigned flags, void *stream);
int ceed_schwarz_destroy(ceed_schwarz_t sw);

/* ---------------------------------------------------------------- adjoint */

/* Geometric factor without coefficient, Ghat = w adj(J) adj(J)^T / det J (6 per point, FP64),
 * stored for the adjoint: same size/layout as diffusion qdata in F64.  Synchronizes. */
int ceed_build_geometry(ceed_mesh_t mesh, void *geo, void *stream);

/* y = A(k) x for a per-point coefficient k (device [n_elem][Q^3], caller's element order),
 * with geometry either stored (geo from ceed_build_geometry) or recomputed from the vertices
 * (geo = NULL).  FP64; with CEED_APPLY_F64_DF (stored geometry only) the same result to FP64
 * accuracy from double-float arithmetic on the FP32 pipe (compensated sums).  nrhs/ncomp = 1.
 * Errors: INVALID (unknown flag bits), UNSUPPORTED (CEED_APPLY_F64_DF without stored geometry). */
int ceed_apply_diffusion_k(ceed_mesh_t mesh, const double *k, const void *geo, const double *x,
                           double *y, unsigned flags, void *stream);

/* Adjoint of L = 0.5 ||A(k) x - b||^2 given r = A(k) x - b:
 *   dLdx = A(k) r                                   (A is symmetric)
 *   dLdk[e][q] = (grad_xi r^e)_q^T Ghat_q (grad_xi x^e)_q
 * in one fused kernel per colour.  dLdx: device FP64 [n_ldof]; dLdk: device [n_elem][Q^3]
 * (caller's element order).  geo: stored geometry or NULL (recompute).  flags: 0, or
 * CEED_APPLY_F64_DF (stored geometry only) for the double-float arithmetic. */
int ceed_apply_diffusion_adjoint(ceed_mesh_t mesh, const double *k, const void *geo, const double *x,
                                 const double *r, double *dLdx, double *dLdk, unsigned flags, void *stream);

/* ---------------------------------------------------------------- non-tensor (simplex) elements */

/* Non-tensor elements (paper Section 3, libCEED's non-tensor bases and the MAGMA backend): the
 * caller provides the interpolation and gradient matrices of the basis at the quadrature points and
 * the quadrature weights, and the operator applies them densely, element by element:
 *   mass       y^e = B^T D B u^e,   D = w |det J| rho
 *   diffusion  y^e = G^T D G u^e,   D = w k adj(J) adj(J)^T / det J   (3x3 per point)
 * The operator is basis- and rule-agnostic; the element geometry is the affine simplex map
 * x(xi) = v0 + sum_d xi_d (v_d - v0) from 4 vertices (tetrahedra).  L-vectors are FP64 [n_ldof]
 * (one component).  Two algorithms, selectable per (op, prec):
 *   CEED_NT_FUSED  one fused kernel (gather, forward contraction, pointwise D, transposed
 *                  contraction in shared memory and registers), 32 elements per thread block;
 *   CEED_NT_GEMM   the paper's GEMM formulation: the element inputs form one [E x P] matrix, each
 *                  basis action is one GEMM with the [P x D Q] basis matrix (cuBLAS), optionally
 *                  split into a strided batch of eta-element blocks; gemm_mode 0 = native
 *                  FP64/FP32, 1 = emulated on the tensor cores (FP64: fixed-point slices; FP32:
 *                  three BF16 terms), 2 = TF32 inputs (F32 only; about 1e-3 relative accuracy).
 *   CEED_NT_TC     (F32, P in {4, 10, 20, 35, 56, 84}: the degree-1..6 tetrahedra) one fused kernel on
 *                  the tensor cores (tcgen05): tiles of 128 elements, both basis actions as TF32 matrix
 *                  products with FP32-level accuracy from the three-product split
 *                  a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, the pointwise D on the CUDA cores between them.
 * Precisions: F64, F32 and F64_DF (FP64-accurate on the FP32 pipe: values, tables and quadrature
 * data as double-float pairs, every sum a compensated dot product; FUSED only).
 * All finish with a deterministic transposed restriction (every node sums its element entries in
 * a fixed order).  The handle owns its tables, an element-vector buffer [P][E] and, once the GEMM
 * algorithm has been selected or tuned, two GEMM work arrays ([P][E] and [3 Q][E] doubles). */
typedef struct ceed_nt_s *ceed_nt_t;
typedef enum { CEED_NT_FUSED = 0, CEED_NT_GEMM = 1, CEED_NT_TC = 2 } ceed_nt_algo;

typedef struct {
  int64_t n_elem;            /* E >= 1 */
  int64_t n_ldof;            /* nodes, < 2^29 */
  int32_t P;                 /* basis functions per element, 1..128 */
  int32_t Q;                 /* quadrature points per element, 1..1024 */
  const double *interp;      /* host [Q][P]: B[q][n] = phi_n(xi_q) */
  const double *grad;        /* host [3][Q][P]: G[d][q][n] = d phi_n / d xi_d (xi_q) */
  const double *qweight;     /* host [Q] reference weights (sum = reference volume) */
  const double *qref;        /* host [Q][3] reference coordinates of the points (for x(xi_q)) */
  const int32_t *elem_dofs;  /* device [E][P], node n of element e (the column order of interp/grad) */
  const double *vertices;    /* device [E][4][3] simplex vertices v0..v3 */
  const uint8_t *dirichlet;  /* device [n_ldof] (nonzero = Dirichlet node) or NULL */
} ceed_nt_desc;

/* The degree-p tetrahedron as a basis for ceed_nt_setup (a helper; the operator takes any basis):
 * equispaced Lagrange basis of P_p on the reference tetrahedron {xi >= 0, xi_1+xi_2+xi_3 <= 1}, in
 * Silvester's product form, nodes (i, j, k)/p with i + j + k <= p ordered k slowest and i fastest;
 * the conical product rule with q Gauss-Jacobi points per collapsed direction (exact for total
 * degree 2q - 1; point a + q (b + q c) at xi = (u_a, (1-u_a) v_b, (1-u_a)(1-v_b) w_c)).
 * Sizes: P = (p+1)(p+2)(p+3)/6, Q = q^3; p in 1..7, q in 1..10.  Host arrays, no GPU work. */
int ceed_simplex_sizes(int p, int q, int32_t *P, int32_t *Q);
int ceed_simplex_basis(int p, int q, double *interp, double *grad, double *qweight, double *qref);

/* Build a non-tensor operator handle: copies the basis to the device, validates elem_dofs (in
 * range, no node twice in an element, every node referenced), builds the transposed restriction.
 * Synchronizes `stream`.  Errors: INVALID, OOM, CUDA. */
int ceed_nt_setup(const ceed_nt_desc *desc, ceed_nt_t *out, void *stream);
int ceed_nt_destroy(ceed_nt_t h);
/* Quadrature-data bytes for (op, prec F64, F32 or F64_DF); layout [ncomp][Q][E] (element fastest). */
size_t ceed_nt_qdata_bytes(ceed_nt_t h, int op, int prec);
/* Quadrature data of the affine simplices (coefficients as for ceed_build_qdata; PER_QPT is
 * [E][Q]).  Synchronizes; BAD_GEOMETRY if det J <= 0 in some element. */
int ceed_nt_build_qdata(ceed_nt_t h, int op, int coeff_kind, const double *coeff, int prec, void *qdata,
                        void *stream);
/* y = A x with the algorithm selected for (op, prec) (default FUSED); asynchronous on `stream`;
 * y overwritten; CEED_APPLY_DIRICHLET masks Dirichlet rows and columns (y = x there). */
int ceed_nt_apply(ceed_nt_t h, int op, const void *qdata, int prec, const double *x, double *y,
                  unsigned flags, void *stream);
/* Select the algorithm for (op, prec); GEMM allocates the handle's GEMM work arrays. */
int ceed_nt_set_algorithm(ceed_nt_t h, int op, int prec, int algo, int64_t eta, int gemm_mode);
int ceed_nt_get_algorithm(ceed_nt_t h, int op, int prec, int32_t *algo, int64_t *eta, int32_t *gemm_mode,
                          float *ms);
/* Autotuner (the paper's selection of routine and batch size eta by measurement): times FUSED,
 * TC (F32, supported P) and GEMM with eta in {all, 1024, 4096, 16384, 65536} and gemm_mode 0 and 1
 * (and 2 if include_tf32, F32 only) on the caller's buffers (y overwritten) with CUDA events, and
 * keeps the fastest for (op, prec).  Synchronizes `stream`. */
int ceed_nt_autotune(ceed_nt_t h, int op, const void *qdata, int prec, const double *x, double *y,
                     int include_tf32, void *stream);
/* Synchronizes `stream`; TIMEOUT if a bounded device-side wait of an earlier tensor-core launch
 * expired (the launch then left its element vectors incomplete). */
int ceed_nt_status(ceed_nt_t h, void *stream);

/* ---------------------------------------------------------------- conforming hp (variable order) */

/* Mixed-order elements joined into one continuous space (the mixed-order workload of the batched
 * apply, with conforming interfaces): a structured nx x ny x nz lattice of hexahedra, element
 * e = ex + nx (ey + ny ez) of order orders[e].  Minimum rule: every face and edge carries the lowest
 * order of the elements sharing it; the space is {u continuous, u|_e in Q_{p_e}, u on a face or
 * edge in Q of that entity's order}.  It is the image of a conforming prolongation P from true dofs
 * to element nodes (an element node takes the value of the polynomial of the lowest-dimensional
 * entity it lies on: that entity's GLL Lagrange interpolant, composed through lower-order edges).
 * Operator on true dofs: y = P^T blockdiag(A_e) P x, A_e the element matrices of Section 2 (each
 * order group applied by the fused tensor-product kernels).
 * True-dof numbering: vertices (i, j, k) with i fastest; edges along x, then y, then z, each axis by
 * lower vertex with i fastest, interior nodes in increasing coordinate; faces normal to x, y, z, by
 * lower corner, interior nodes with the lower in-plane axis fastest; element interiors in element
 * order, node a fastest.  Element-node rows (ceed_hp_prolong): order groups by ascending order,
 * elements by ascending index, nodes a + P (b + P c).  The handle owns P, P^T, per-group meshes,
 * quadrature data and two element-vector work arrays. */
typedef struct ceed_hp_s *ceed_hp_t;
typedef struct {
  int32_t nx, ny, nz;          /* elements per direction */
  const int32_t *orders;       /* host [nx ny nz], each in 1..8 */
  const double *vertices;      /* device [E][8][3] trilinear element maps (as for ceed_mesh_desc) */
  int32_t q_rule;              /* GLL (Q = p+1) or GAUSS (Q = p+2), every element */
  int32_t dirichlet;           /* nonzero: the true dofs on the lattice boundary are Dirichlet dofs */
} ceed_hp_desc;
/* The space alone, on the host (no GPU work): for the lattice and orders (host [nx ny nz], 1..8)
 * of an hp description, the true-dof count, the element-node row count and the nonzeros of P; when
 * row_ptr, col, val and dirichlet are all given (else all NULL), also the CSR of P (row_ptr
 * [n_rows + 1], col [nnz], val [nnz]; rows as for ceed_hp_prolong) and dirichlet [n_true] (1 on the
 * lattice boundary).  The same construction ceed_hp_setup uploads.  Errors: INVALID, OOM. */
int ceed_hp_prolongation(int32_t nx, int32_t ny, int32_t nz, const int32_t *orders, int64_t *n_true,
                         int64_t *n_rows, int64_t *nnz, int64_t *row_ptr, int64_t *col, double *val,
                         uint8_t *dirichlet);
/* Build the space (host) and the per-order meshes.  Synchronizes `stream`.  Errors: INVALID, OOM, CUDA. */
int ceed_hp_setup(const ceed_hp_desc *desc, ceed_hp_t *out, void *stream);
int ceed_hp_destroy(ceed_hp_t h);
/* Number of true dofs, of element-node rows, of order groups. */
int ceed_hp_info(ceed_hp_t h, int64_t *n_true, int64_t *n_rows, int32_t *n_groups);
/* Quadrature data of every order group (handle-owned) for (op, prec F64, F32 or F64_DF: the
 * FP64-accurate double-float element kernels); coefficients ONE, CONST or SINE.  Synchronizes
 * `stream`. */
int ceed_hp_build_qdata(ceed_hp_t h, int op, int coeff_kind, const double *coeff, int prec, void *stream);
/* Element vectors u_elem = P x (device FP64 [n_rows]); asynchronous. */
int ceed_hp_prolong(ceed_hp_t h, const double *x, double *u_elem, void *stream);
/* y = P^T A P x on true dofs (device FP64 [n_true]); `prec` selects the quadrature data and the
 * arithmetic of the element kernels; CEED_APPLY_DIRICHLET masks the Dirichlet dofs.  Asynchronous. */
int ceed_hp_apply(ceed_hp_t h, int op, int prec, const double *x, double *y, unsigned flags, void *stream);

/* ---------------------------------------------------------------- vectors */

/* Deterministic dot product of two device FP64 vectors; the result is written to *out
 * (device FP64).  work: device scratch of ceed_dot_workspace_bytes(n) bytes. */
size_t ceed_dot_workspace_bytes(int64_t n);
int ceed_dot(const double *x, const double *y, int64_t n, double *out, void *work, void *stream);

/* Dot product that performs no device allocation and needs no workspace argument.
 * The paper has no counterpart; this entry point exists for callers that cannot allocate
 * device memory: a solver library that receives only vector pointers from a host application
 * which owns all device memory through its own pool, or an iteration loop where cudaMalloc and
 * cudaFree are unacceptable because they can stall or synchronize the device, or can fail midway
 * through a solve when memory is tight.
 * Scratch: a static device array of 32768 FP64 partial sums (256 KiB) that every GPU which loads
 * the library holds until the process exits.  Each block sums a fixed chunk of 8192 entries, so
 * n may be at most ceed_dot_noalloc_max_n() = 268,435,456; larger n returns CEED_ERR_INVALID
 * (use ceed_dot with a workspace instead).  The result is deterministic for a given n; it can
 * differ from ceed_dot's in the last bits because the chunking differs.
 * The first call on a device looks up the scratch address on that device (cudaGetSymbolAddress
 * with the device current); make that first call before any stream capture.  All calls share the
 * one array and each call overwrites the slots it reads, so nothing has to be cleared, but calls
 * that may overlap on the GPU (different streams, no ordering between them) race on the scratch
 * and must be serialized by the caller.  x, y: device FP64 [n]; out: device FP64 scalar. */
int64_t ceed_dot_noalloc_max_n(void);
int ceed_dot_noalloc(const double *x, const double *y, int64_t n, double *out, void *stream);

/* ---------------------------------------------------------------- status, limits, measurement */

/* Synchronizes `stream` and reports whether a bounded device wait of an earlier apply on this mesh
 * gave up (the TMA copy of an element's quadrature data did not land within the wait limit): then
 * it clears the flag and returns CEED_ERR_TIMEOUT, and the y of those applies is incomplete
 * (elements whose wait gave up write nothing).  CEED_OK otherwise. */
int ceed_mesh_status(ceed_mesh_t mesh, void *stream);

/* Limits of the bounded device-side waits (not an operation of the paper; failure handling):
 * copy_polls governs each apply kernel's wait for its quadrature-data copy (negative: the default
 * bound of 2^22 polls; 0: give up at once; the kernels keep that bound a compile-time constant, so
 * other values are INVALID), barrier_polls the grid barriers of the persistent batched launch and of
 * the fused CG iteration (negative: the default 2^25 polls; 0 .. 2^25: that many polls).  A wait
 * that runs out records CEED_ERR_TIMEOUT (read by ceed_mesh_status / ceed_batch_status, returned by
 * ceed_cg_solve) and the kernel finishes without hanging; tests use 0 to drive these paths.
 * Process-wide; applies to launches issued afterwards (a batch's CUDA graph keeps the limits it was
 * captured with: re-create the batch or re-run ceed_batch_autotune to pick up new ones). */
int ceed_set_wait_limits(int64_t copy_polls, int64_t barrier_polls);

/* Arithmetic-throughput measurement (not an operation of the paper; it gives the operators'
 * roofline denominators): kind 0 = FP64 FMA, 1 = FP32 FMA, 2 = packed two-lane FP32 FMA
 * (fma.rn.f32x2).  Runs independent FMA chains on every SM (64 warps per SM, about 50-100 ms per
 * run, best of three) on `stream` and returns TFLOP/s (2 flops per FMA), FMAs per clock per SM and
 * the SM clock in MHz seen by one block during the run (either pointer may be NULL).  Kinds 3 and
 * 4 run the double-float operator's packed compensated sums instead (4 independent Dot2
 * accumulators per thread, each step a TwoProduct with cross terms and a TwoSum in two-lane form)
 * at 16 warps per SM (that operator's occupancy) and 64; they return FP32 lane operations per second
 * / 1e12 in *tflops and lane operations per clock per SM in *fma_per_clk_sm.  Synchronizes
 * `stream`.  Errors: INVALID, CUDA. */
int ceed_fma_throughput(int kind, double *tflops, double *fma_per_clk_sm, double *sm_mhz, void *stream);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char *ceed_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CEED_GB300_H */
