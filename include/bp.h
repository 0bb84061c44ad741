/*
 * bp.h -- C ABI of libbp: first-order (Blatter-Pattyn) Stokes velocity assembly and Newton
 * solve on extruded wedge meshes, for NVIDIA B300 (sm_103a).
 *
 * The operations follow arXiv 2204.04321 ("Performance portable ice-sheet modeling with
 * MALI"):
 *   - Sec. 2, Eq. FOStokes / effvisc / effeps: the momentum equations
 *       -div(2 mu eps_1) + rho g ds/dx = 0,  -div(2 mu eps_2) + rho g ds/dy = 0,
 *     Glen viscosity mu = 1/2 A^(-1/n) (eps_e^2 + delta)^((1-n)/(2n)) (delta regularises U = 0),
 *     a stress-free surface, the linear sliding (Robin) law 2 mu eps . n + beta u = 0 at the bed
 *     and, on the vertical margins, either stress-free or the ocean condition (bp_params.margin);
 *     A constant or a nodal field (Arrhenius relation, bp_mesh_set_rate_factor);
 *   - Sec. 3.1, Eq. residual: low-order nodal prismatic (6-node wedge) finite elements on the
 *     3D mesh extruded from a base triangulation give the residual F(U; {phi_i}, {grad phi_i}, H, beta);
 *   - Sec. 3.1, Eq. linearsystem: damped Newton J delta = -F, U <- U + alpha delta;
 *   - Sec. 3.2: the Jacobian is the exact derivative of the residual (forward-mode automatic
 *     differentiation in the paper), scattered into a sparse matrix.
 *
 * Fixed discretisation (part of the ABI): reference wedge lambda = (1 - xi - eta, xi, eta),
 * N = lambda_a (1 -/+ zeta)/2, 3-point triangle rule x 2-point Gauss in zeta (6 points),
 * basal face with the same triangle rule over the true (3D) face area.
 *
 * Degrees of freedom are column-major and interleaved: for base vertex a, node level
 * l = 0..L (0 = bed) and component c (0 = u, 1 = v): dof = 2 * (a * (L + 1) + l) + c.
 * The Jacobian is stored in CSR over all structurally coupled pairs (base vertices equal or
 * sharing a triangle, |l - l'| <= 1, all four component pairs), columns sorted, explicit zeros
 * kept.  Row pointers are int64, column indices int32.
 *
 * Conventions for every call:
 *   - the return value is a bp_status (0 = success);
 *   - device buffers U, R, J are owned by the caller; the mesh object owns the mesh arrays,
 *     the sparsity pattern and all scratch it needs, all on the device current at upload;
 *   - velocity arrays U_dev must be 16-byte aligned (the kernels load (u, v) pairs together);
 *   - Jacobian value arrays must be 8-byte aligned (FP32 values are scattered as (u, v) pairs);
 *   - calls that take a stream are asynchronous on that stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream) unless documented as synchronising;
 *   - residual / Jacobian outputs are overwritten, never accumulated;
 *   - units are m, yr, Pa; no rescaling happens inside the library;
 *   - there is no CPU fallback: every computation runs in the library's CUDA kernels.
 */
#ifndef BP_H
#define BP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BP_OK = 0,
  BP_EINVAL = 1,    /* a NULL pointer, a size out of range or an unknown option */
  BP_EMESH = 2,     /* invalid mesh: bad index, non-positive area or thickness, sigma not increasing */
  BP_ENOMEM = 3,    /* device allocation failed */
  BP_ECUDA = 4,     /* a CUDA runtime call failed */
  BP_ENAN = 5,      /* a non-finite value was met */
  BP_ENOCONV = 6,   /* an iteration limit was reached before the tolerance */
  BP_EUNSUP = 7,    /* a parameter combination the kernels do not implement (e.g. n != 3) */
  BP_ESIZE = 8,     /* the problem exceeds a fixed capacity of the call (see BP_NOALLOC_MAX_NDOF) */
  BP_EIO = 9        /* a file could not be read or written, or is not in the expected format */
} bp_status;

/* Lateral margin condition (paper Sec. 2, third boundary condition, on the vertical faces over the
 * boundary edges of the base triangulation):
 *   BP_MARGIN_FREE   2 mu eps_c . n = 0 (natural; the default reading for land-terminating margins);
 *   BP_MARGIN_OCEAN  2 mu eps_c . n = (rho g (s - z) - rho_w g max(-z, 0)) n_c: the cryostatic ice
 *                    pressure of the first-order model against the ocean's back-pressure below sea
 *                    level z = 0 (the paper prints max(z, 0), read as the submerged part max(-z, 0)).
 *                    In weak form R_i gets -int_face (rho g (s - z) - rho_w g max(-z, 0)) n_c N_i, a
 *                    solution-independent load formed once at upload with a 2 x 2 Gauss rule per face
 *                    (two points along the edge, two in zeta). */
enum { BP_MARGIN_FREE = 0, BP_MARGIN_OCEAN = 1 };

/* Glen exponent n (must be 3: the kernels take the cube root of eps_e^2 + delta), rate factor
 * A [Pa^-n yr^-1] (> 0; see bp_mesh_set_rate_factor for a field), ice density rho [kg m^-3],
 * gravity g [m s^-2], regularisation delta [yr^-2]. */
typedef struct {
  double n, A, rho, g, delta;
  double rho_w;      /* sea-water density (kg m^-3), read with BP_MARGIN_OCEAN */
  int32_t margin;    /* BP_MARGIN_FREE or BP_MARGIN_OCEAN */
  int32_t reserved;
} bp_params;

/* Host description of an extruded mesh; all arrays are read during bp_mesh_upload only. */
typedef struct {
  int32_t nv;           /* base vertices */
  int32_t ntri;         /* base triangles */
  int32_t nlayers;      /* L >= 1 element layers, L + 1 node levels */
  int32_t reserved;
  const double* xy;     /* [nv][2] horizontal coordinates (m) */
  const int32_t* tri;   /* [ntri][3] vertex indices, counter-clockwise */
  const double* bed;    /* [nv] bed elevation b (m) */
  const double* thick;  /* [nv] ice thickness H > 0 (m); node z = b + sigma_l H, surface s = b + H */
  const double* beta;   /* [nv] sliding coefficient >= 0 (Pa yr m^-1) */
  const double* sigma;  /* [nlayers + 1] 0 = sigma_0 < ... < sigma_L = 1 */
  bp_params params;
} bp_mesh_desc;

typedef struct bp_mesh bp_mesh; /* opaque, library-owned */

typedef struct {
  int64_t ndof;        /* 2 nv (L + 1) */
  int64_t nnz;         /* 4 (nv + 2 E)(3 L + 1), E = base edges */
  int64_t nwedges;     /* ntri * L */
  int32_t nv, ntri, nlayers, ncolors; /* ncolors: triangle colours of the coloured scatter */
  int64_t device_bytes; /* device memory held by the mesh object */
} bp_mesh_info_t;

/* Jacobian precision of the derivative lanes (the residual is FP64 except with BP_F32_ALL, and
 * FP64-accurate double-single with the _DS kinds):
 *   BP_F64   native FP64 lanes;
 *   BP_F32   FP32 lanes (J values are float);
 *   BP_F64X2 FP64-accurate lanes built from pairs of FP32 numbers (hi + lo, error-free sum and
 *            product transformations, relative error ~2^-46 per operation); J values are double;
 *            Jacobian assembly only, sum-factorised method only.  It moves the lane arithmetic to
 *            the FP32 pipe (~60x the FP64 rate on B300); the rank-one part of the element matrix
 *            is applied in a loop over the quadrature points whose factors wait in shared memory.
 *   BP_F32_DS   FP32 lanes with a double-single value path: the quadrature-point arithmetic of the
 *            residual and of the viscosity in pairs of FP32 numbers (~2^-47 per operation; the
 *            inverse cube root from an FP32 seed and one pair correction), the per-column and
 *            per-level geometry in FP64.  R is FP64-accurate (same parity bar as BP_F64); J values
 *            are float.  Sum-factorised method only.
 *   BP_F64X2_DS paired lanes and the double-single value path: residual and Jacobian FP64-accurate
 *            with the quadrature-point arithmetic on the FP32 pipe; J values are double.
 *            Sum-factorised method only; no Picard matrix.
 *   BP_F32_ALL  FP32 lanes and an FP32 value path: the geometry, the 2D velocity gradients and the
 *            vertical velocity differences are formed in FP64 and rounded once, everything at the
 *            quadrature points (strain rates, viscosity, stresses, element residual) runs in FP32.
 *            J values are float; R is still a double array but carries FP32 rounding (relative
 *            ~1e-7 of the element contributions).  Sum-factorised method only.  Meant for the
 *            early steps of an inexact Newton solve (bp_solve_opts.value32_rtol), where the
 *            residual is far above that rounding. */
enum { BP_F64 = 0, BP_F32 = 1, BP_F64X2 = 2, BP_F32_ALL = 3, BP_F32_DS = 4, BP_F64X2_DS = 5 };
/* Scatter of element contributions: atomics, or colour by colour with plain read-modify-write. */
enum { BP_SCATTER_AUTO = 0, BP_SCATTER_ATOMIC = 1, BP_SCATTER_COLOR = 2 };
/* How the element Jacobian is formed: forward-mode dual numbers with 12 lanes (one per
 * element dof), or the same tangent sum-factorised over the extruded quadrature. */
enum { BP_JAC_AUTO = 0, BP_JAC_DUAL = 1, BP_JAC_FACTORED = 2 };

/* Library version string (static storage). */
const char* bp_version(void);
/* Human-readable text of a status code (static storage). */
const char* bp_strerror(int status);

/*
 * Validate the mesh, build the extruded CSR pattern, the per-triangle scatter slots, the
 * triangle colouring and the solution-independent data (driving-stress load vector,
 * basal friction matrices), and copy everything to the current device.  Mirrors the paper's
 * memoisation (Sec. 4.1): data that do not change between Newton iterations are formed once.
 * Synchronises `stream` before returning.  On error *out is NULL and nothing is leaked.
 * Errors: BP_EINVAL (NULL pointers, nv/ntri/nlayers < 1), BP_EMESH (index out of range,
 * clockwise or degenerate triangle, H <= 0, beta < 0, sigma not strictly increasing from 0 to 1),
 * BP_EUNSUP (n != 3), BP_ENOMEM, BP_ECUDA.
 */
int bp_mesh_upload(const bp_mesh_desc* desc, void* stream, bp_mesh** out);

/* Free a mesh (NULL is a no-op).  Synchronises the device. */
void bp_mesh_free(bp_mesh* mesh);

/* Sizes of an uploaded mesh. */
int bp_mesh_info(const bp_mesh* mesh, bp_mesh_info_t* info);

/* Borrowed device pointers to the CSR pattern (valid until bp_mesh_free):
 * rowptr [ndof + 1] int64, colidx [nnz] int32. */
int bp_csr_pattern(const bp_mesh* mesh, const int64_t** rowptr_dev, const int32_t** colidx_dev);

/*
 * Residual R(U) (Eq. residual), FP64.  U_dev, R_dev: device arrays of ndof doubles in the
 * dof order above; R is overwritten.  Asynchronous on `stream`.
 * Errors: BP_EINVAL (NULL arguments), BP_ECUDA (launch failure).
 */
int bp_assemble_residual(bp_mesh* mesh, const double* U_dev, double* R_dev, void* stream);

/*
 * Jacobian dR/dU at U (Sec. 3.2) into J_vals_dev ([nnz] values on the bp_csr_pattern
 * pattern: double for BP_F64 and BP_F64X2, float for BP_F32 and BP_F32_ALL) and, if R_dev != NULL,
 * the residual (FP64; FP32-accurate with BP_F32_ALL).
 * Both outputs are overwritten (zeroing is part of the call).  `scatter` is a BP_SCATTER_*,
 * `method` a BP_JAC_*.  Asynchronous on `stream`.
 * Errors: BP_EINVAL (NULL U/J, misaligned U/J, unknown precision/scatter/method), BP_EUNSUP (BP_F64X2 or
 * BP_F32_ALL with BP_JAC_DUAL), BP_ENOMEM (first call with R_dev == NULL allocates a residual
 * scratch in the mesh object), BP_ECUDA.
 */
int bp_assemble_jacobian(bp_mesh* mesh, const double* U_dev, double* R_dev, void* J_vals_dev,
                         int precision, int scatter, int method, void* stream);

/* ------------------------------------------------------------------------------------------
 * Solver (Sec. 3.1 Eq. linearsystem, Sec. 3.3 / 4.4).  All vectors are device arrays of ndof
 * doubles in the dof order above.  The entry points of this section (and the initial guesses and
 * energies below) take meshes of at most 64 layers and answer BP_EUNSUP for more; the assembly
 * has no layer limit.
 * ------------------------------------------------------------------------------------------ */

/*
 * y = J x for a Jacobian on the bp_csr_pattern pattern (J_vals_dev: double for BP_F64, float for
 * BP_F32 or BP_F32_ALL; products and sums in FP64).  The operator application "Op*x" of the linear solve.
 * J, x and y must be 16-byte aligned (u and v rows are processed as pairs).  Asynchronous.
 * Errors: BP_EINVAL (NULL, misaligned, unknown precision), BP_ECUDA.
 */
int bp_spmv(bp_mesh* mesh, const void* J_vals_dev, int precision, const double* x_dev, double* y_dev,
            void* stream);

/*
 * y = J x with FP32 values, FP32 vectors and FP32 products and sums: the product of the mixed-
 * precision Krylov solves and MDSC cycles (the same kernel they run).  J (float values on the
 * bp_csr_pattern pattern), x and y (ndof floats each, dof order) are caller-owned device arrays,
 * 16-byte aligned.  Asynchronous.  Errors: BP_EINVAL (NULL or misaligned), BP_EUNSUP (more than 64
 * layers), BP_ECUDA.
 */
int bp_spmv_f32(bp_mesh* mesh, const float* J_vals_dev, const float* x_dev, float* y_dev, void* stream);

/*
 * Vertical-line preconditioner: for every base vertex, the block-tridiagonal part of J that
 * couples the (L + 1) levels of its column (2 x 2 blocks) is factorised by block Thomas elimination
 * without pivoting (J is symmetric positive definite), one thread per column -- the per-vertical-line
 * batched LU of the paper's semicoarsening prolongation (Sec. 4.4).  bp_colprec_setup factorises
 * and keeps the factors in the mesh: FP64 arithmetic and factors for a BP_F64 Jacobian, FP32
 * arithmetic and factors for a BP_F32 (or BP_F32_ALL) Jacobian (the mixed-precision Krylov path),
 * which bp_colprec_apply then applies in FP32 arithmetic.  bp_colprec_apply computes z = P^-1 r.  Asynchronous.
 * Errors: BP_EINVAL, BP_ENOMEM (workspace), BP_ECUDA.
 */
int bp_colprec_setup(bp_mesh* mesh, const void* J_vals_dev, int precision, void* stream);
int bp_colprec_apply(bp_mesh* mesh, const double* r_dev, double* z_dev, void* stream);

/*
 * Matrix-dependent semicoarsening (MDSC) two-level preconditioner (Sec. 4.4: the vertical-line
 * prolongation of the paper's multigrid, then a 2D solve of the plane problem), one symmetric cycle:
 *   P      semicoarsening to the top level: in each column the top value is extended downwards by
 *          the harmonic extension of the column's block-tridiagonal part T of J (the column rows
 *          below the top satisfied with zero right-hand side), from T's block-Thomas factors;
 *   A_c    = P^T J P on the base vertices (2 x 2 blocks over the closed neighbourhoods);
 *   B_c    8 steps of Chebyshev acceleration of block-Jacobi on A_c over [lam / 30, lam], lam the
 *          Gershgorin bound of D^-1 A_c (D its diagonal blocks);
 *   S      = 0.7 T^-1 (the damped vertical-line solve);
 *   z1 = S r;  z2 = z1 + P B_c P^T (r - J z1);  z = z2 + S (r - J z2)  (symmetric positive definite).
 * bp_mdsc_setup also sets up the column factors (as bp_colprec_setup) and reads the Gershgorin
 * bound back (synchronises `stream`); precision as for bp_colprec_setup (FP32 arithmetic for an
 * FP32 Jacobian).  bp_mdsc_apply computes z = M^-1 r (device arrays of ndof doubles, 16-byte
 * aligned) with the Jacobian values J_vals_dev that bp_mdsc_setup saw (the cycle multiplies by J);
 * asynchronous.  Errors: BP_EINVAL (NULL, misaligned, unknown precision, no setup), BP_ENOMEM,
 * BP_ENAN (non-finite plane operator), BP_ECUDA.
 */
int bp_mdsc_setup(bp_mesh* mesh, const void* J_vals_dev, int precision, void* stream);
int bp_mdsc_apply(bp_mesh* mesh, const void* J_vals_dev, const double* r_dev, double* z_dev, void* stream);

/*
 * The MDSC cycle with the plane problem solved by smoothed-aggregation algebraic multigrid (paper
 * Sec. 4.4 and Sec. 3.1: semicoarsening to one layer, then AMG in 2D with a Chebyshev smoother):
 * the cycle of bp_mdsc_setup with B_c = one V-cycle on A_c:
 *   aggregation of each level's block graph (pattern of A_k, 2 x 2 blocks): vertices in order, a
 *     vertex whose whole neighbourhood is free starts an aggregate of that neighbourhood; then each
 *     vertex still free joins the first-pass aggregate of its lowest-numbered such neighbour;
 *   P_k = (I - 4 / (3 lam_k) D_k^-1 A_k) Pt_k, Pt_k(i, agg(i)) = I (the two translations);
 *   A_{k+1} = P_k^T A_k P_k; levels until <= 64 vertices (at most 8 levels; coarsening stops when a
 *     level shrinks by less than 0.8); the coarsest solved with its dense inverse (<= 512 vertices);
 *   V-cycle: 3 Chebyshev block-Jacobi steps over [lam_k / 30, lam_k] from zero, coarse correction,
 *     the same polynomial on the new residual (symmetric positive definite).
 * The aggregates and patterns depend on the mesh only and are built on the host at the first setup
 * of the mesh; each setup then forms the levels on the device.  bp_mdsc_amg_setup synchronises
 * `stream` (it reads the level-0 Gershgorin bound back); bp_mdsc_amg_apply is asynchronous.
 * bp_mdsc_amg_levels writes the vertex count of each level (at most max_levels) and the number of
 * levels; bp_mdsc_amg_aggregates copies the aggregate index of every vertex of level `level`
 * (0 .. levels - 2) to host memory.
 * Errors: BP_EINVAL (NULL, misaligned, unknown precision, no setup, level out of range),
 * BP_EUNSUP (coarsest level above 512 vertices), BP_ENOMEM, BP_ENAN, BP_ECUDA.
 */
int bp_mdsc_amg_setup(bp_mesh* mesh, const void* J_vals_dev, int precision, void* stream);
int bp_mdsc_amg_apply(bp_mesh* mesh, const void* J_vals_dev, const double* r_dev, double* z_dev, void* stream);
int bp_mdsc_amg_levels(const bp_mesh* mesh, int32_t* sizes_host, int max_levels, int* nlevels);
int bp_mdsc_amg_aggregates(const bp_mesh* mesh, int level, int32_t* agg_host);

/*
 * Discrete energy Pi_h(U) = sum_q w det J A^(-1/n) 2n/(n+1) (eps_e^2 + delta)^((n+1)/(2n))
 * + sum_i load_i U_i + 1/2 sum_bed U_b^T M_beta U_b, whose gradient is the residual (same
 * quadrature).  Not written in the paper: it follows from Eq. effvisc / effeps and is the merit
 * function of the damped Newton line search.  Writes the value to *out_host; synchronises `stream`.
 */
int bp_energy(bp_mesh* mesh, const double* U_dev, double* out_host, void* stream);

/*
 * Energy change Pi_h(U + alpha D) - Pi_h(U), formed term by term as differences (the stress term
 * through the exact expansion of eps_e^2 in alpha and a^2 - b^2 = (a - b)(a + b) on cube roots),
 * so it stays accurate when it is far below the rounding level of Pi_h itself -- the quantity the
 * Newton line search compares.  Writes *out_host; synchronises `stream`.
 */
int bp_energy_change(bp_mesh* mesh, const double* U_dev, const double* D_dev, double alpha, double* out_host,
                     void* stream);

/*
 * The same energy change in the arithmetic of one of the Newton solve's line searches: BP_F64 (as
 * bp_energy_change), BP_F64X2_DS (the per-point work in double-single pairs on the FP32 pipe,
 * FP64-accurate: the line search of the BP_F64 and BP_F64X2_DS solves), or BP_F32 (the per-point
 * work in FP32 with the per-column geometry and the driving and basal terms in FP64: the line
 * search of the mixed-precision solves; ~1e-5 relative).  Inputs as for bp_energy_change.
 * Errors: BP_EINVAL (NULL pointer, another precision), BP_ENOMEM, BP_ECUDA.
 */
int bp_energy_change_ex(bp_mesh* mesh, const double* U_dev, const double* D_dev, double alpha, int precision,
                        double* out_host, void* stream);

/* Initial guesses of the Newton solve (not in the paper). */
enum { BP_GUESS_ZERO = 0, BP_GUESS_SIA = 1 };
/*
 * U = 0, or the shallow-ice + linear-sliding profile
 *   u(z) = -(2A/(n+1)) (rho g)^n |grad s|^(n-1) grad s (H^(n+1) - (s - z)^(n+1)) - rho g H grad s / beta
 * with the nodal grad s = area-weighted mean of the P1 gradients of the adjacent triangles
 * (beta = 0 at a vertex gives the non-sliding profile).  Asynchronous.
 */
int bp_initial_guess(bp_mesh* mesh, int kind, double* U_dev, void* stream);

enum { BP_KRYLOV_CG = 0, BP_KRYLOV_GMRES = 1 };
/* Preconditioner of the Newton solve's CG (bp_solve_opts.preconditioner). */
enum { BP_PREC_COLUMN = 0, BP_PREC_MDSC = 1, BP_PREC_MDSC_AMG = 2 };
/* Line search of bp_newton_solve (bp_solve_opts.line_search). */
enum { BP_LS_OFF = 0, BP_LS_HALVING = 1, BP_LS_QUADRATIC = 2 };

typedef struct {
  double rtol;        /* stop when ||F(U)||_2 <= rtol ||F(0)||_2 (F(0) is the driving-stress load) */
  int max_newton;     /* Newton iteration limit (<= 64) */
  int max_krylov;     /* Krylov iterations per Newton step */
  double eta_max;     /* Eisenstat-Walker forcing term cap (choice 2, gamma = 0.9) */
  int precision;      /* BP_F64: FP64 Jacobian and Krylov, the line search's energy change
                         FP64-accurate in double-single pairs (bp_energy_change_ex); BP_F32: FP32
                         Jacobian lanes and Krylov (inexact Newton), FP32 energy change; the
                         residual, viscosity, norms and update stay FP64.
                         BP_F64X2_DS: FP64-accurate residual and Jacobian from the double-single value
                         path and paired lanes, FP64 Krylov, the line search's energy change in pairs
                         (no Picard steps); BP_F32_DS: as BP_F32 with the double-single value path
                         (residual FP64-accurate) */
  int krylov;         /* BP_KRYLOV_CG (default: the Jacobian is SPD), or BP_KRYLOV_GMRES: restarted
                         GMRES(gmres_restart) as the paper's Krylov method, right-preconditioned by
                         the column solve (classical Gram-Schmidt twice; the Hessenberg problem on the
                         host, one synchronisation per iteration), a cross-check of CG */
  int line_search;    /* Armijo test on the energy change (c = 1e-4, at most 11 trials), a BP_LS_*:
                         BP_LS_OFF full steps; BP_LS_HALVING alpha = 1, 1/2, ..., 2^-10;
                         BP_LS_QUADRATIC backtracking by quadratic interpolation of the energy
                         change, each new alpha kept within [0.1, 0.9] of the rejected one */
  int check_every;    /* batch replays (device_loop 0, or no conditional graph nodes): convergence
                         is read back every check_every iterations */
  double picard_rtol; /* > 0: while ||F|| > picard_rtol ||F(0)|| take Picard steps (the Jacobian
                         without the eta' rank-one part: the fixed-viscosity matrix, SPD, cheaper
                         to assemble), then Newton steps; 0: Newton from the first step */
  double value32_rtol; /* BP_F32 only, > 0: while ||F|| > value32_rtol ||F(0)|| assemble with
                          BP_F32_ALL (FP32 value path: an inexact residual, rounding ~1e-7 of the
                          element contributions), then with the FP64 value path; a residual that
                          comes out below value32_rtol ||F(0)|| is assembled again with the FP64
                          value path before it is tested, so convergence is always tested on an
                          FP64 residual.  0: FP64 value path throughout; values in (0, rtol) are
                          refused (BP_EINVAL): an FP32 residual could then pass the test */
  int device_loop;    /* 1: the CG iterations run as a device-driven loop (a conditional WHILE graph
                         node, 4 iterations per pass, programmatic launches): the device stops the
                         loop, no host check in between; 0: replays of a captured 8-iteration batch
                         with a host check every check_every iterations */
  int preconditioner; /* BP_PREC_COLUMN: the vertical-line block solve; BP_PREC_MDSC: the two-level
                         semicoarsening cycle (bp_mdsc_setup); BP_PREC_MDSC_AMG: the same cycle with
                         the SA-AMG plane solve (bp_mdsc_amg_setup); with device_loop 0 their iterations
                         are launched from the host, one host check each (CG only: BP_EUNSUP with
                         GMRES) */
  int gmres_restart;  /* GMRES restart length m, 1..64 (default 50; the basis holds m + 1 vectors) */
} bp_solve_opts;

typedef struct {
  int newton_iters;          /* Newton steps taken */
  int krylov_iters;          /* total Krylov iterations */
  int converged;             /* 1 if ||F|| <= rtol ||F(0)|| */
  int value32_steps;         /* steps assembled with the FP32 value path (bp_solve_opts.value32_rtol) */
  double fnorm_ref;          /* ||F(0)||_2 */
  double fnorm_initial;      /* ||F(U_0)||_2 */
  double fnorm_final;        /* ||F(U)||_2 at return */
  double history[65];        /* ||F(U_k)|| / ||F(0)|| for k = 0..newton_iters */
  int krylov_per_newton[64];
  double alpha[64];          /* accepted damping factors */
  double t_total, t_assemble, t_precond, t_krylov, t_linesearch; /* seconds (CUDA events) */
} bp_solve_report;

/* Defaults: rtol 1e-8, 50 Newton, 1000 Krylov, eta_max 0.1, BP_F64, CG, line search on, check 8,
 * picard_rtol 0, value32_rtol 0, device_loop 1, BP_PREC_COLUMN, gmres_restart 50. */
void bp_solve_opts_default(bp_solve_opts* opts);

/*
 * Damped Newton (Eq. linearsystem) from the guess in U_dev to ||F|| <= rtol ||F(0)||: per step
 * the Jacobian and residual are assembled (bp_assemble_jacobian; the Picard matrix instead while
 * opts->picard_rtol asks for it), the column preconditioner is factorised, J delta = -F is solved
 * by preconditioned CG to the Eisenstat-Walker tolerance, and the step length alpha is the first
 * trial of opts->line_search with the energy change (bp_energy_change_ex in the solve's line-search
 * arithmetic: pairs for BP_F64 and BP_F64X2_DS, FP32 for BP_F32 and BP_F32_DS) at (U, delta, alpha)
 * <= 1e-4 alpha F . delta
 * (Armijo on the energy; the last trial is taken if none passes).  After a full step that reduced
 * the residual tenfold (the quadratic regime) the next full step is taken without the test.
 * U_dev holds the last iterate on return.
 * Synchronises `stream`.  Errors: BP_EINVAL, BP_ENOMEM, BP_ECUDA, BP_ENAN (non-finite residual, or a
 * non-finite Krylov residual: the solve stops at once),
 * BP_ENOCONV (max_newton reached; the report is filled either way).
 */
int bp_newton_solve(bp_mesh* mesh, double* U_dev, const bp_solve_opts* opts, bp_solve_report* report,
                    void* stream);

/* ------------------------------------------------------------------------------------------
 * Ensemble assembly: many uneven meshes in one persistent launch.
 * ------------------------------------------------------------------------------------------ */
typedef struct bp_ensemble bp_ensemble; /* opaque */

/*
 * Bind `count` uploaded meshes (all on the current device) to their caller-owned buffers:
 * U_dev[i] (input, ndof_i doubles), R_dev[i] (output residual, ndof_i doubles) and J_dev[i]
 * (output Jacobian values, nnz_i of `precision`); pointer arrays are host arrays, read here only.
 * The Jacobian uses the sum-factorised lanes.  Members are not copied: they must outlive the
 * ensemble.  Errors: BP_EINVAL (NULL, count < 1, meshes on another device), BP_ENOMEM, BP_ECUDA.
 */
int bp_ensemble_create(bp_mesh* const* members, int count, const double* const* U_dev, double* const* R_dev,
                       void* const* J_dev, int precision, void* stream, bp_ensemble** out);

/*
 * Autotuner: times every candidate -- columns per thread block in {32, 64, 128, 256} times scatter
 * mode {atomic: one persistent launch over a (member, tile) queue; coloured: one persistent launch
 * per colour over all members' tiles of that colour} -- as the median of `reps` runs, keeps the
 * fastest and captures the whole assembly (zero-initialisation + launches) in a CUDA graph.
 * times_ms[8] (nullable) receives the medians in the order cpb-major, atomic then coloured;
 * chosen[2] (nullable) receives (columns per block, scatter).  Synchronises `stream`.
 */
int bp_ensemble_tune(bp_ensemble* ens, int reps, void* stream, double* times_ms, int* chosen);

/* Use the given candidate (cpb in {32, 64, 128, 256}, scatter BP_SCATTER_ATOMIC or
 * BP_SCATTER_COLOR) instead of tuning: captures its graph.  Synchronises `stream`. */
int bp_ensemble_select(bp_ensemble* ens, int cpb, int scatter, void* stream);

/*
 * Assemble the residuals and Jacobians of all members (overwriting them): replays the tuned graph,
 * or launches the default candidate (128 columns per block, atomic) if bp_ensemble_tune has not
 * run.  Asynchronous on `stream`.
 */
int bp_ensemble_assemble(bp_ensemble* ens, void* stream);

/* Free the ensemble (not its members).  Synchronises the device. */
void bp_ensemble_free(bp_ensemble* ens);

/* ------------------------------------------------------------------------------------------
 * Learned warm start (not in the paper): a per-column MLP 16 -> 128 -> 128 -> 128 -> 32 (ReLU)
 * mapping column features to the 2 (L + 1) = 22 level velocities of a 10-layer column.
 * BF16 operands, FP32 accumulation, on the 5th-generation tensor cores (tcgen05, TMEM).
 * ------------------------------------------------------------------------------------------ */
#define BP_MLP_IN 16
#define BP_MLP_HIDDEN 128
#define BP_MLP_OUT 32
#define BP_MLP_OUT_USED 22   /* (u, v) at 11 node levels */
#define BP_MLP_LEVELS 11
typedef struct bp_mlp bp_mlp; /* opaque */

/* Number of FP32 parameters: [W1 (128x16), b1, W2 (128x128), b2, W3 (128x128), b3, W4 (32x128), b4],
 * weights row-major (out x in). */
int64_t bp_mlp_param_count(void);
/* New network on the current device, He-uniform weights from a counter-based generator
 * (SplitMix64 of seed and parameter index), zero biases, fresh Adam state. */
int bp_mlp_create(uint64_t seed, bp_mlp** out);
void bp_mlp_free(bp_mlp* mlp);
/* Copy the FP32 master parameters to / from host memory (n = bp_mlp_param_count()); setting resets
 * Adam.  Synchronise `stream`. */
int bp_mlp_get_params(const bp_mlp* mlp, float* host, int64_t n, void* stream);
int bp_mlp_set_params(bp_mlp* mlp, const float* host, int64_t n, void* stream);
/* Y[n][32] = MLP(X[n][16]); X is BF16 (raw uint16 bits), Y FP32.  Asynchronous. */
int bp_mlp_forward(bp_mlp* mlp, const uint16_t* X_dev, int64_t n, float* Y_dev, void* stream);
/* Loss (1/n) sum_rows sum_{j < 22} (Y - T)^2 and its gradient (FP32, parameter layout above,
 * overwritten in grad_dev) for X[n][16] (BF16), T[n][32] (FP32).  *loss_host (nullable) receives
 * the loss and makes the call synchronous.  Errors: BP_EINVAL, BP_ENOMEM, BP_ECUDA. */
int bp_mlp_gradient(bp_mlp* mlp, const uint16_t* X_dev, const float* T_dev, int64_t n, float* grad_dev,
                    double* loss_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the gradient of the batch; asynchronous. */
int bp_mlp_train_step(bp_mlp* mlp, const uint16_t* X_dev, const float* T_dev, int64_t n, float lr,
                      void* stream);
/* Write / read the FP32 master parameters as a NumPy .npy file (format 1.0: a little-endian
 * float32 vector of bp_mlp_param_count() entries, the layout above), so numpy.save / numpy.load
 * exchange the same files.  Loading resets Adam (as bp_mlp_set_params) and accepts .npy versions
 * 1.0-3.0 whose header describes exactly that vector.  Synchronous (default stream).
 * Errors: BP_EINVAL (NULL), BP_EIO (file not readable / writable, or another array), BP_ECUDA. */
int bp_mlp_save(const bp_mlp* mlp, const char* path);
int bp_mlp_load(bp_mlp* mlp, const char* path);
/* Column features X[nv][16] (BF16) of an uploaded 10-layer mesh, built from the quantities
 * q = (ln(H / 1000 m), asinh(1000 s_x) / 4, asinh(1000 s_y) / 4, ln(beta / 1000)) with the nodal
 * grad s (area-weighted as for the shallow-ice guess): [0..7] hi/lo BF16 splits of the local q
 * (about 16 significant bits), [8..11] q averaged over closed neighbourhoods in 8 sweeps (~5 km),
 * [12..14] ln beta, s_x, s_y terms after 40 sweeps (~15 km), [15] sigma_1 (the layering).
 * Errors: BP_EUNSUP if the mesh does not have 10 layers. */
int bp_mlp_features(bp_mesh* mesh, uint16_t* X_dev, void* stream);
/* Replace beta on an uploaded mesh (host array [nv]) and rebuild the basal friction matrices. */
int bp_mesh_set_beta(bp_mesh* mesh, const double* beta_host, void* stream);
/*
 * Temperature-dependent rate factor (Sec. 2, the Arrhenius relation A = A0 exp(-Q / (R T*))):
 * A_host [nv][L + 1] (node (a, l) at a (L + 1) + l, Pa^-3 yr^-1, > 0), e.g. evaluated from a
 * pressure-corrected temperature field.  The library keeps the nodal hardness B = A^(-1/3) and
 * interpolates it at the quadrature points with the wedge basis (2 mu = B (eps_e^2 + delta)^(-1/3));
 * the residual, the Jacobian, the energy and every solver call use it.  A_host = NULL restores the
 * uniform A of bp_mesh_upload.  Set it before bp_ensemble_create (an ensemble copies the pointer).
 * The shallow-ice initial guess keeps the uniform A.  Synchronises `stream`.
 * Errors: BP_EINVAL (NULL mesh, a value <= 0 or not finite), BP_ENOMEM, BP_ECUDA.
 */
int bp_mesh_set_rate_factor(bp_mesh* mesh, const double* A_host, void* stream);
/* How bp_initial_guess_learned decides between the network's guess and the shallow-ice guess:
 *   BP_JUDGE_RESIDUAL  keep the guess with the smaller FP64 residual norm;
 *   BP_JUDGE_ENERGY    keep the guess with the smaller discrete energy Pi_h (the functional
 *                      Newton minimises: Pi_h(U) - Pi_h(U*) ~ 1/2 |U - U*|^2 in the Jacobian's norm),
 *                      decided by the sign of the FP64-accurate energy change from the shallow-ice
 *                      guess to the network's (bp_energy_change_ex with BP_F64X2_DS);
 *   BP_JUDGE_NONE      always keep the network's guess (evaluation). */
enum { BP_JUDGE_RESIDUAL = 0, BP_JUDGE_ENERGY = 1, BP_JUDGE_NONE = 2 };
/*
 * Learned initial guess: per column and component c the network scales the sliding part
 * b_c = u_sia,c(bed) and the deformation part d_c = u_sia,c - b_c of the shallow-ice profile,
 * u_c = (1 + y_2c) b_c + (1 + y_2c+1) d_c, which keeps the vertical profile consistent (vertical
 * shear dominates the stress on thin layers) and reduces to the shallow-ice guess where the network
 * has learned nothing; written in the dof order.  Falls back to the shallow-ice guess when that one
 * wins under `judge` (a BP_JUDGE_*; the FP64 residual by default); *used (nullable) receives 1 if the
 * network's prediction was kept, 0 otherwise.  Synchronises `stream`.
 * Errors: BP_EINVAL (NULL, misaligned U, unknown judge), BP_EUNSUP (mesh without 10 layers),
 * BP_ENOMEM, BP_ECUDA.
 */
int bp_initial_guess_learned(bp_mesh* mesh, bp_mlp* mlp, double* U_dev, int judge, int* used, void* stream);
/*
 * The structured decoder of bp_initial_guess_learned on its own: U_dev [ndof] (dof order,
 * 16-byte aligned) = decoder(Y_dev, shallow-ice guess) for network outputs Y_dev [nv][32] (FP32;
 * entries 0..3 of each column are read: y_b,u, y_d,u, y_b,v, y_d,v), for any layer count.
 * The shallow-ice guess is computed into library-owned workspace.  Asynchronous.
 * Errors: BP_EINVAL (NULL, misaligned U), BP_ENOMEM, BP_ECUDA.
 */
int bp_learned_decode(bp_mesh* mesh, const float* Y_dev, double* U_dev, void* stream);
/*
 * The decoder's training targets for a velocity field U_dev (a Newton solution, dof order): per
 * column and component c the scales (s_b, s_d) of the shallow-ice sliding part b_c and deformation
 * part d_c that minimise |s_b b + s_d d - u|^2 + reg^2 (|b|^2 (s_b - 1)^2 + |d|^2 (s_d - 1)^2) over the
 * column's levels (FP64 2 x 2 normal equations; a numerically singular column keeps s = 1),
 * written as T_dev[a][0..3] = s - 1 clipped to [-5, 5] (FP32; T_dev[a][4..31] = 0), [nv][32].
 * Asynchronous.  Errors: BP_EINVAL (NULL, misaligned U, reg < 0 or not finite), BP_ENOMEM, BP_ECUDA.
 */
int bp_learned_targets(bp_mesh* mesh, const double* U_dev, double reg, float* T_dev, void* stream);

/*
 * Measured FMA throughput of the current device (the roofline denominator of the assembly, which
 * is bound by the FP64 pipe; the paper names no such figure): a kernel of 8 independent FMA chains
 * per thread, 64 warps per SM on every SM, best of 5 timed launches after a warm-up (CUDA events
 * on `stream`), 2 flops per FMA.  precision: BP_F64 (DFMA) or BP_F32 (FFMA).  Allocates and frees a
 * small output buffer; synchronises `stream`.  Errors: BP_EINVAL, BP_ENOMEM, BP_ECUDA.
 */
int bp_measure_fma_peak(int precision, double* tflops, void* stream);

/*
 * Allocation-free variant of bp_assemble_jacobian (R not returned).  The paper has no
 * counterpart: this entry point exists for callers that must not allocate device memory once
 * running (a fixed device-memory budget, or a host framework whose allocator owns all device
 * memory), for whom the residual scratch that bp_assemble_jacobian allocates on its first call
 * with R_dev == NULL is not acceptable.  Its residual scratch is a fixed array inside the
 * library of BP_NOALLOC_MAX_NDOF doubles (8 MiB), which every GPU that loads the library holds
 * until the process exits; the call itself performs no allocation.
 *   - J_vals_dev, precision, scatter, method: as for bp_assemble_jacobian; J is overwritten.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.  The address is
 *     kept for the life of the process: do not use this entry point after cudaDeviceReset on that
 *     device (the library's module, and with it the array, may then be loaded at a new address).
 *   - All calls share the one array and leave their residual in it; each call starts it afresh.
 *     Calls whose executions overlap on the GPU (different streams, or different meshes on the
 *     same device at the same time) race on the array: serialise them.
 * Errors: BP_ESIZE if the mesh has more than BP_NOALLOC_MAX_NDOF degrees of freedom,
 * BP_EINVAL (NULL U/J, unknown precision/scatter/method), BP_ECUDA.
 */
#define BP_NOALLOC_MAX_NDOF 1048576
int bp_assemble_jacobian_noalloc(bp_mesh* mesh, const double* U_dev, void* J_vals_dev, int precision,
                                 int scatter, int method, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BP_H */
