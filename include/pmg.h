/*
 * pmg.h -- C ABI of the GB300 (sm_103a) p-multigrid-preconditioned Krylov solver for the
 * pressure-Poisson problem of the sigma-mapped nodal spectral element wave model of
 * Melander, Laskowski, Sherwin & Engsig-Karup (arXiv 2411.14977).
 *
 * Problem (the same-geometry symmetric reading of the paper's Poisson BVP, Sec. 3.1-3.2):
 *   find p in V_P (continuous, degree <= P per quad, Sec. 4) with p = p_D on the free
 *   surface and a(N_i, p) = b_i for every free node i, where
 *     a(v, p) = int_Omega grad v . grad p dOmega, pulled back to the sigma-domain
 *               sigma = (z + h)/d, d = eta + h (Sec. 2.2, Eq. for sigma_x, sigma_z),
 *   on a structured mesh of cells_x x cells_z quadrilaterals (Sec. 4.3) with
 *   Legendre-Gauss-Lobatto nodes and LGL collocation quadrature.
 *
 * Node numbering (every vector in this ABI):  g = ix * NZ + iz,  z fastest.
 *   NZ = cells_z * order + 1, iz = 0 at the bottom, iz = NZ - 1 on the free surface;
 *   NX = cells_x * order + 1 (walls at x0, x1) or cells_x * order (periodic in x).
 *   The free surface row is Dirichlet; walls and bottom are Neumann.
 *
 * Memory: every "_dev" pointer is a CUDA device pointer owned by the caller; every
 *   "_host" pointer is host memory owned by the caller.  The handle owns its workspace
 *   (allocated in pmg_create, freed in pmg_destroy).  Vectors are FP64 unless the name
 *   says f32.  Calls are asynchronous on the given stream (a cudaStream_t passed as
 *   void*, NULL = legacy default stream) unless stated otherwise.
 * Errors: every call returns a pmg_status; no exception crosses the ABI; the message of
 *   the last failure on the calling thread is returned by pmg_last_error().
 * Threads: one handle must not be used by two threads at once.  Calls on one handle
 *   that overlap on the GPU (different streams) race on its workspace.
 */
#ifndef PMG_H_
#define PMG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PMG_OK = 0,
  PMG_ERR_INVALID = 1,        /* bad descriptor, option, pointer or size                  */
  PMG_ERR_OOM = 2,            /* device or pinned-host allocation failed (nothing leaked)  */
  PMG_ERR_CUDA = 3,           /* a CUDA runtime call failed                                */
  PMG_ERR_NOT_CONVERGED = 4,  /* iteration cap reached; last iterate and info are filled   */
  PMG_ERR_NONFINITE = 5,      /* NaN/Inf in the input or in the residual                   */
  PMG_ERR_TIMEOUT = 6         /* a bounded device-side wait gave up                        */
} pmg_status;

/* precision of the V-cycle (preconditioner); the outer residual and result are FP64 */
enum { PMG_FP64 = 0, PMG_MIXED_FP32 = 1, PMG_MIXED_BF16 = 2 };
/* outer method (always FP64 on the actual-geometry operator):
 *   PMG_PCG  preconditioned CG (with a mixed-precision V-cycle: flexible CG)
 *   PMG_FCG  flexible CG (Polak-Ribiere beta)
 *   PMG_PDC  preconditioned defect correction x <- x + B(b - Ax) (Sec. 5.4)
 *   PMG_IR   FP64 iterative refinement around an inner FP32 flexible-CG solve
 *            (mixed precision only; inner_max / inner_tol apply)
 *   PMG_GMRES  flexible GMRES(gmres_restart) with the V-cycle as right preconditioner
 *            (Sec. 5.4's GMRES-MG on the same-stage operator); Arnoldi by classical
 *            Gram-Schmidt applied twice on the device, one host synchronisation per
 *            restart cycle
 * With PMG_MIXED_FP32 the V-cycle B runs in FP32 on the FP32-rounded residual.
 * PMG_MIXED_BF16 (requires PMG_IR): as PMG_MIXED_FP32, and the inner solve's
 * actual-geometry operator runs its contractions on the BF16 tensor cores with hi/lo
 * split operands and FP32 accumulation (pmg_apply_bf16, split = 1). */
enum { PMG_PCG = 0, PMG_FCG = 1, PMG_PDC = 2, PMG_IR = 3, PMG_GMRES = 4 };
/* smoother: element-block additive Schwarz (Sec. 5.3), blocks inverted by fast
 * diagonalisation (exact for the separable flat-geometry level operators) */
enum { PMG_ASM_FDM = 0, PMG_ASM_DENSE = 1 };
/* geometry the multigrid levels are built on: the flat, linearised (eta = 0) geometry
 * that makes the preconditioner time-constant (Sec. 5.4) */
enum { PMG_ACTUAL = 0, PMG_FLAT_LINEARISED = 1 };

typedef struct {
  double x0, x1;     /* horizontal extent of the tank                                     */
  double h;          /* still-water depth (flat bottom z = -h)                            */
  int cells_x;       /* quads in x (>= 1; >= 3 and a power of two when periodic_x)         */
  int cells_z;       /* quads in sigma (>= 1)                                              */
  int order;         /* polynomial order P along x, 1..10                                  */
  int periodic_x;    /* 0: walls at x0, x1 (Neumann); 1: periodic in x                    */
  int order_z;       /* polynomial order along sigma (Sec. 5.1); 0 = order.  Different orders
                        are semi-coarsened (the higher one reduced by the level rule, not below
                        the other, until they match) and are built for the pairs of the
                        paper's scaling study: order_z = 8 with order 2..10                   */
} pmg_mesh_desc;

typedef struct {
  int precision;     /* PMG_FP64 | PMG_MIXED_FP32 | PMG_MIXED_BF16                          */
  int outer;         /* PMG_PCG | PMG_FCG | PMG_PDC | PMG_IR                                */
  int smoother;      /* PMG_ASM_FDM (fast diagonalisation) | PMG_ASM_DENSE (dense inverses of
                        the (P+1+2o)^2-node subdomain blocks, built on the device, Sec. 5.3) */
  int precond_geom;  /* PMG_FLAT_LINEARISED (time-constant levels on eta = 0, Sec. 5.4) |
                        PMG_ACTUAL (every level but the order-1 one re-discretised on the
                        current surface at each pmg_set_geometry; needs PMG_ASM_DENSE, equal
                        orders and a constant depth)                                        */
  int overlap;       /* Schwarz overlap in node lines (0 or 1)                              */
  int nu;            /* pre- and post-smoothing sweeps per level (>= 1)                     */
  double omega;      /* smoother damping                                                    */
  double tol;        /* stop when ||b~ - A p||_2 <= tol ||b~||_2 over free nodes            */
  int max_iter;      /* outer iteration cap                                                 */
  int inner_max;     /* mixed precision: inner FCG iteration cap per refinement step        */
  double inner_tol;  /* mixed precision: inner relative residual target                     */
  int nlevels;       /* 0 = the paper's coarsening rule; else level_orders[0..nlevels-1]    */
  int level_orders[8];
  int fuse_residual; /* sweeps (FP32) and restrictions that form their own level residual:  */
                     /* 1 on every level, 0 (default) never, -1 where pmg_autotune measured   */
                     /* it to be 10% faster (solve times are equal within noise at config 2) */
  int flat_kernel;   /* FP32 level operator: 0 slab CTAs (one element column each), 1 one   */
                     /* thread per node, 2 tiled CTAs (one thread per element; constant-depth */
                     /* levels of equal orders up to 8, others slab) of 16 element columns x  */
                     /* 8 element rows, or a tiled shape given as 10000 + 100 EXT + ZT (EXT   */
                     /* columns of 8, 16 or 32, ZT rows of 4 or 8, EXT ZT a multiple of 32 and */
                     /* at most 256), 3 slab CTAs of 256 threads whose inputs are staged by   */
                     /* TMA bulk copies (constant depth, equal orders, 16-byte-aligned        */
                     /* vectors; others slab), or that shape with 1000 + threads (64..512,   */
                     /* whole warps), -1 (default) slab until pmg_autotune picks by time     */
  int df64_outer;    /* outer actual-geometry operator (FP64 vectors in and out) computed in */
                     /* double-float arithmetic on the FP32 pipe (48-bit significand): 1 on, */
                     /* 0 off (FP64 pipe), -1 (default) on for the mixed precisions only     */
  int gmres_restart; /* PMG_GMRES cycle length m, 1..60 (default 30); the handle then holds */
                     /* 2m+1 extra FP64 vectors                                              */
  int sweep_kernel;  /* FP32 Schwarz sweep (constant depth, equal orders): 0 slab CTAs (one  */
                     /* element column each), 1 z-split CTAs (zc element rows of one element */
                     /* column each, halo elements recomputed, slabs staged by TMA bulk      */
                     /* copies), -1 (default) slab until pmg_autotune picks by time, or a    */
                     /* z-split shape 1000 zc + threads (zc 1..64, threads 32..256, whole warps) */
  int fuse_coarse;   /* mixed precisions: the FP32 V-cycle's levels of order <= 4 and the    */
                     /* coarse solve run as one cooperative launch (grid barriers between    */
                     /* the steps, bounded waits: PMG_ERR_TIMEOUT): 1 on where the levels    */
                     /* qualify (flat constant-depth levels of equal orders, fast-diagonal-   */
                     /* isation smoother), 0 off (one launch per step), -1 (default) off    */
                     /* until pmg_autotune measures the fused V-cycle faster                  */
} pmg_opts;

typedef struct {
  int iterations;        /* outer iterations (PCG/FCG/PDC) or refinement steps (mixed)      */
  int inner_iterations;  /* mixed precision: total inner FCG iterations                    */
  double rel_residual;   /* final ||b~ - A p||_2 / ||b~||_2, FP64                          */
  double seconds;        /* wall time of the call                                          */
  int status;            /* pmg_status of the solve                                         */
} pmg_solve_info;

typedef struct pmg_handle pmg_handle;

/* Fill *opts with the defaults: FP64, PCG, FDM-ASM, flat preconditioner, overlap 1, nu 2,
 * omega 0.8, tol 1e-10, max_iter 500, inner_max 40, inner_tol 1e-5, paper level rule,
 * autotuned kernel families (flat_kernel, sweep_kernel -1), split level residuals,
 * double-float outer operator for the mixed precisions, GMRES restart 30, fused coarse
 * V-cycle where pmg_autotune finds it faster (fuse_coarse -1). */
void pmg_default_opts(pmg_opts* opts);

/* ---- host-only queries (no device work; they run without a GPU) ---------------------- */
/* The level orders pmg_create builds for (mesh, opts): the coarsening rule P_{n-1} =
 * ceil((P_n+1)/2) down to 2, then 1 (Sec. 5.1), the semi-coarsening pairs when
 * mesh->order_z differs from mesh->order (the higher order steps by the rule, not below
 * the other, until they match), or opts->level_orders.  *nlevels receives the count;
 * orders and orders_z (each NULL or room for 16 ints, caller-owned) receive the orders
 * along x and sigma, finest first.  opts NULL = defaults.  Validates mesh and opts exactly
 * as pmg_create does: PMG_ERR_INVALID with pmg_last_error() set on bad input. */
pmg_status pmg_level_sequence(const pmg_mesh_desc* mesh, const pmg_opts* opts, int* nlevels, int* orders,
                              int* orders_z);
/* The reference-element tables the setup uses for order p, 1 <= p <= 10 (Sec. 4.3): LGL
 * nodes (p+1, ascending) and weights (p+1); the nodal derivative matrix D, row-major
 * (p+1) x (p+1) with D[i][m] = dh_m/dr at node i; and for 1 <= pc <= p the interpolation
 * J that takes order-pc nodal values to the order-p nodes (the prolongation's 1D factor,
 * Sec. 5.2), row-major (p+1) x (pc+1); pc = 0 skips J.  Any output pointer may be NULL
 * (host memory, caller-owned).  PMG_ERR_INVALID for p or pc out of range. */
pmg_status pmg_basis_tables(int p, int pc, double* nodes, double* weights, double* D, double* J);
/* The fast-diagonalisation factors of one additive-Schwarz element class (Sec. 5.3) as the
 * setup builds them for a level of order p (1..10) and overlap o (0 or 1).  The 1D
 * subdomain is an element's p+1 node lines plus o lines of each neighbour, cut at walls,
 * on a canonical line of unit-reference cells; along sigma (dir = 1) the surface line is
 * Dirichlet and left out.  cls: 0 interior element, 1 first (wall / bottom), 2 last
 * (wall / surface), 3 both (a single element).  With K the assembled 1D LGL stiffness
 * (sum over cells of D^T diag(w) D) and M the assembled weights, restricted to the k
 * nodes present: V (row-major NB x NB, NB = p+1+2o; row = local node, column = mode; rows
 * of absent nodes and columns past k zero) has V^T M V = I and V^T K V = diag(lam); lam
 * has NB entries, zero past k.  Host-only; caller-owned host buffers.  PMG_ERR_INVALID
 * for arguments out of range or NULL outputs. */
pmg_status pmg_schwarz_class(int p, int o, int dir, int cls, double* V, double* lam, int* k);

/* Build the mesh, the level hierarchy P_{n-1} = ceil((P_n+1)/2) down to 2, then 1
 * (Sec. 5.1), the transfer matrices I = Phi V^-1 (Sec. 5.2), the Schwarz factors
 * (Sec. 5.3) and the coarse factor, on the current CUDA device; geometry starts flat
 * (eta = 0).  Synchronous.  *out is NULL on failure. */
pmg_status pmg_create(const pmg_mesh_desc* mesh, const pmg_opts* opts, pmg_handle** out);
/* Frees everything pmg_create allocated (device and host); NULL is a no-op.  Lifecycle
 * only: no counterpart in the paper. */
pmg_status pmg_destroy(pmg_handle* h);

/* Sizes of the nodal mesh (the global numbering of Sec. 4.3): total nodes n = NX*NZ, free
 * (non-Dirichlet) nodes, NX, NZ, number of levels (Sec. 5.1).  Any pointer may be NULL. */
pmg_status pmg_num_nodes(const pmg_handle* h, int64_t* n, int64_t* n_free, int* nx, int* nz,
                         int* nlevels);
/* Order and node counts of level l (0 = finest) of the hierarchy of Sec. 5.1.
 * PMG_ERR_INVALID for a bad level. */
pmg_status pmg_level_info(const pmg_handle* h, int level, int* order, int* nx, int* nz);
/* Launch configuration of level l's FP32 kernels as set at creation or chosen by
 * pmg_autotune: flat32 = level operator (> 0 slab CTA size, < 0 node-parallel CTA size,
 * >= 10000 tiled shape 10000 + 100 EXT + ZT, see pmg_opts.flat_kernel), fdm32 = Schwarz
 * sweep (< 1000: slab CTA size; >= 1000: z-split with fdm32 / 1000 element rows and
 * fdm32 % 1000 threads per CTA), xfer = transfer CTA size.  Host-side read; any pointer may be NULL.
 * The paper has no counterpart.  PMG_ERR_INVALID for a bad handle or level. */
pmg_status pmg_level_kernels(const pmg_handle* h, int level, int* flat32, int* fdm32, int* xfer);
/* Fused coarse V-cycle (pmg_opts.fuse_coarse): *first_level = the first level it covers
 * (its steps run from there down to the order-1 coarse solve and back up in one
 * cooperative launch; -1 when the levels do not qualify), *on = 1 while the FP32 V-cycle
 * uses it, *threads and *ctas_per_sm = its launch shape, us[0], us[1] = the FP32 V-cycle's
 * microseconds without and with it as pmg_autotune timed them (0 before tuning).  The
 * paper has no counterpart (a V-cycle step per launch, or many, computes the same Sec. 5
 * V-cycle).  Host-side read; any pointer may be NULL.  PMG_ERR_INVALID for a bad handle. */
pmg_status pmg_fused_vcycle_info(const pmg_handle* h, int* first_level, int* on, int* threads, int* ctas_per_sm,
                                 float* us);
/* Switches the fused coarse V-cycle on (1) or off (0) for the following solves and
 * V-cycles, as pmg_autotune leaves it otherwise.  PMG_ERR_INVALID when on = 1 and the
 * levels do not qualify (pmg_fused_vcycle_info: first_level = -1). */
pmg_status pmg_set_fused_vcycle(pmg_handle* h, int on);
/* x* of every node column (NX values) and sigma of every node row (NZ values) of the
 * sigma-domain mesh (Sec. 2.2, LGL nodes per cell, Sec. 4.3); caller-owned host arrays. */
pmg_status pmg_node_coords(const pmg_handle* h, double* x_cols_host, double* sigma_rows_host);

/* Per-stage geometry (Sec. 2.2): eta at every node column (NX values, device).  The
 * surface is the degree-P interpolant of these values per cell; d = eta + h must stay
 * positive.  The multigrid hierarchy is not rebuilt (flat preconditioner, Sec. 5.4). */
pmg_status pmg_set_geometry(pmg_handle* h, const double* eta_dev, void* stream);
/* Mixed-stage operator (Sec. 3, the mixed-stage Laplace operator nabla^k . nabla^(k-1)):
 * sets the stage-k geometry as pmg_set_geometry does (eta: stage k, also used by the
 * right-hand sides) and makes the outer operator a(v, p) = int over the stage-k domain of
 * grad^k v . grad^(k-1) p, the trial gradient taken on the stage-(k-1) surface eta_prev
 * (both NX doubles, device).  Nonsymmetric: pmg_solve then needs outer PMG_PDC or
 * PMG_GMRES (else PMG_ERR_INVALID); the V-cycle keeps the flat geometry.
 * pmg_set_geometry returns to the same-stage operator. */
pmg_status pmg_set_geometry_mixed(pmg_handle* h, const double* eta_dev, const double* eta_prev_dev, void* stream);

/* Varying still-water depth h(x) (Sec. 2.2, the sigma map sigma = (z + h(x)) / d with
 * d = eta + h(x); Sec. 6 runs over a submerged bar): h_dev holds the depth at every node
 * column (NX doubles, device, each > 0 and finite; the bottom is the degree-P interpolant
 * per cell).  It replaces the mesh's constant h for every later operator, load vector and
 * solve: the outer operator gains the bottom-slope metric terms, the bottom Neumann term
 * uses the arc length of the mapped bottom, and every multigrid level becomes the
 * still-water operator with the slope terms dropped -- each node column keeps its depth,
 * evaluated at the level's nodes -- which is still a Kronecker sum, so the Schwarz blocks
 * (now one x-factorisation per element column) and the coarse solve stay exact.  The
 * geometry set last is recomputed.  Synchronous on `stream` (tables are built on the host).
 * PMG_ERR_INVALID: NULL, a depth <= 0 or non-finite (also after interpolation to a coarse
 * level), the BF16 tensor-core operator (PMG_MIXED_BF16), a periodic mesh of one cell.
 * Gradient recovery (pmg_gradient) then uses the depth and its slope too.  Afterwards
 * pmg_set_geometry_mixed returns PMG_ERR_INVALID (the mixed-stage operator takes a constant
 * depth only); there is no way back to a constant depth but a new handle. */
pmg_status pmg_set_bathymetry(pmg_handle* h, const double* h_dev, void* stream);

/* The load of the pressure Poisson problem (Sec. 3.1-3.2: Dirichlet on the free surface,
 * Neumann on walls and bottom) in the weak form of Sec. 4.2:
 * b_i = -int N_i f dOmega + int_{Gamma_N} N_i g dGamma (LGL collocation), b = 0 on the
 * free surface.  f: nodal values (n); g_bottom: outward normal derivative on the bottom
 * per node column (NX); g_left / g_right: on the walls per node row (NZ).  Any g may be
 * NULL (zero flux); the wall arrays are ignored when periodic. */
pmg_status pmg_assemble_rhs(pmg_handle* h, const double* f_dev, const double* g_bottom_dev,
                            const double* g_left_dev, const double* g_right_dev, double* b_dev,
                            void* stream);
/* b_i = scale * int grad N_i . (u, w) dOmega: the weak divergence of a nodal velocity
 * field (the right-hand side rho/dt div u* of the pressure step, Sec. 3.1, in the weak form
 * of Sec. 4.2; it carries n.u on walls and bottom). */
pmg_status pmg_assemble_rhs_div(pmg_handle* h, const double* u_dev, const double* w_dev,
                                double scale, double* b_dev, void* stream);

/* Solve for the pressure (Sec. 5: the outer iteration of Sec. 5.4 preconditioned by one
 * p-multigrid V-cycle): p_out = p_D on the free surface, A_FF p_F = b_F - A_FD p_D.
 * b_dev: load vector (free entries used); p_dirichlet_dev: values read on the surface
 * row only; x0_dev: initial guess or NULL (zero).  Returns PMG_ERR_NOT_CONVERGED with the
 * last iterate in p_out when max_iter is hit.  info may be NULL.  Synchronises the stream
 * (the convergence test reads device scalars). */
pmg_status pmg_solve(pmg_handle* h, const double* b_dev, const double* p_dirichlet_dev,
                     const double* x0_dev, double* p_out_dev, pmg_solve_info* info,
                     void* stream);

/* pmg_solve (Sec. 5) with all five vectors in host memory (n doubles each, x0 may be NULL): copies
 * the inputs from the caller's host buffers into device vectors owned by the handle, solves,
 * and copies the pressure back, all on `stream`; returns after the stream has synchronised.
 * Page-locked (pinned) host buffers give asynchronous copies at the full link rate. */
pmg_status pmg_solve_host(pmg_handle* h, const double* b_host, const double* p_dirichlet_host,
                          const double* x0_host, double* p_out_host, pmg_solve_info* info,
                          void* stream);
/* ||b~ - A x~||_2 on the device: x~ is x with its surface row replaced by p_D (the lifted
 * residual that the solve's tolerance is measured in: the residual r of Sec. 5.4 after
 * the Dirichlet lifting).  Synchronises `stream`
 * and writes the norm to *norm (host).  PMG_ERR_NONFINITE for a non-finite input. */
pmg_status pmg_residual_norm(pmg_handle* h, const double* b, const double* p_dirichlet, const double* x,
                             double* norm, void* stream);

/* ---- component entry points (parity tests and benchmarks) ------------------------- */
/* y = A_FF x on free nodes, y = x on the surface row; actual geometry, FP64 (Sec. 4.2). */
pmg_status pmg_apply(pmg_handle* h, const double* x_dev, double* y_dev, void* stream);
/* The same operator (Sec. 4.2) in FP32 storage and arithmetic (the paper computes in FP64). */
pmg_status pmg_apply_f32(pmg_handle* h, const float* x_dev, float* y_dev, void* stream);
/* The same FP32 operator with its four sum-factorised contractions on the BF16 tensor
 * cores (mma.sync m16n8k16, FP32 accumulation): split = 0 rounds D and the operand to
 * BF16 once; split = 1 adds hi*hi + hi*lo + lo*hi of their BF16 hi/lo parts (about 16
 * significant bits per product).  Not in the paper.  x, y: NX*NZ floats on the device. */
pmg_status pmg_apply_bf16(pmg_handle* h, const float* x_dev, float* y_dev, int split, void* stream);
/* Flat level-l operator (the multigrid level matrix of Sec. 5.1 on the linearised geometry
 * of Sec. 5.4), masked like pmg_apply.
 * f32 = 0: FP64 vectors, 1: FP32 vectors. */
pmg_status pmg_level_apply(pmg_handle* h, int level, const void* x_dev, void* y_dev, int f32,
                           void* stream);
/* One additive-Schwarz sweep x += omega W sum_e R_e^T A_e^-1 R_e r (post = 0) or its adjoint
 * (post = 1) on level `level` for a given residual r (Sec. 5.3): a single kernel launch,
 * for timing and tests.  Vectors as in pmg_level_smooth. */
pmg_status pmg_level_sweep(pmg_handle* h, int level, const void* r, void* x, int post, int f32, void* stream);
/* nu Schwarz sweeps on level l for A_l x = b, updating x in place (Sec. 5.3);
 * post = 0: x += omega W sum R^T A_i^-1 R r, post = 1: the adjoint (W applied to r).
 * f32 = 0: FP64 vectors, 1: FP32 vectors (level l's node count each). */
pmg_status pmg_level_smooth(pmg_handle* h, int level, const void* b_dev, void* x_dev, int post,
                            int f32, void* stream);
/* r_c = P^T r_f (level l -> l+1) and x_f += P x_c (level l+1 -> l) (Sec. 5.2). */
pmg_status pmg_restrict(pmg_handle* h, int level, const void* rf_dev, void* rc_dev, int f32,
                        void* stream);
pmg_status pmg_prolong(pmg_handle* h, int level, const void* xc_dev, void* xf_dev, int f32,
                       void* stream);
/* Exact FP64 solve of the coarsest (order 1) level system (free nodes; surface row 0).  The
 * paper names order 1 as the coarsest level (Sec. 5.1) but not its solver. */
pmg_status pmg_coarse_solve(pmg_handle* h, const double* b_dev, double* x_dev, void* stream);
/* z = B r: one V-cycle of the preconditioner on the finest level (Sec. 5). */
pmg_status pmg_vcycle(pmg_handle* h, const void* r_dev, void* z_dev, int f32, void* stream);

/* ---- time-stepper support (the wave-tank workload around the pressure solve) --------- */
/* Nodal physical gradient (d/dx, d/dz) of a nodal field on the current geometry by the
 * lumped-mass L2 projection (the paper's gradient recovery, Sec. 4): element-local
 * derivatives through the sigma-map (Sec. 2.2), averaged over the elements of a node. */
pmg_status pmg_gradient(pmg_handle* h, const double* f_dev, double* fx_dev, double* fz_dev, void* stream);
/* Exponential cut-off filter of the modal coefficients (Sec. "Spectral Filtering"):
 * S(k) = 1 for k <= cutoff, exp(alpha ((k - cutoff)/(P + 1 - cutoff))^beta) above, on the
 * orthonormal Legendre modes of each element, F = V diag(S) V^-1.  pmg_set_filter builds
 * F on the host (0 <= cutoff <= P, alpha <= 0, beta > 0; PMG_ERR_INVALID otherwise).
 * pmg_filter applies F (x) F per element to a nodal field (surface = 0: N values) or F to
 * the surface elevation (surface = 1: NX values) and takes the mean at nodes shared by
 * elements; `out` must not alias `f`. */
pmg_status pmg_set_filter(pmg_handle* h, int cutoff, double alpha, double beta);
pmg_status pmg_filter(pmg_handle* h, const double* f, double* out, int surface, void* stream);
/* eta_x per node column (NX) of the current surface polynomial, the slope in the kinematic
 * condition and the sigma-map (Sec. 2.2, Sec. 4.1); the mean at element edges. */
pmg_status pmg_surface_slope(pmg_handle* h, double* etax_dev, void* stream);
/* Explicit forcing of the inviscid momentum equations with the static pressure folded in
 * (p = p_D + rho g (eta - z), Sec. 2.1): Fu = -(u u_x + w u_z) - g eta_x, Fw = -(u w_x + w w_z).
 * The dynamic pressure then solves Delta p_D = rho div F with p_D = 0 on the surface and
 * d p_D/dn = rho n.F elsewhere: pmg_assemble_rhs_div(Fu, Fw, rho). */
pmg_status pmg_forcing(pmg_handle* h, const double* u_dev, const double* w_dev, const double* ux_dev,
                       const double* uz_dev, const double* wx_dev, const double* wz_dev, const double* etax_dev,
                       double g, double* Fu_dev, double* Fw_dev, void* stream);
/* Stage rates at fixed sigma: eta_t = w - u eta_x on the surface (kinematic condition,
 * Eq. freesurf1); du/dt = F - grad p_D / rho + sigma eta_t du/dz (mesh velocity sigma eta_t),
 * the same for w.  deta has NX entries. */
pmg_status pmg_stage_rates(pmg_handle* h, const double* u_dev, const double* w_dev, const double* uz_dev,
                           const double* wz_dev, const double* Fu_dev, const double* Fw_dev, const double* px_dev,
                           const double* pz_dev, const double* etax_dev, double rho, double* du_dev, double* dw_dev,
                           double* deta_dev, void* stream);
/* out = y + a x over n doubles: the stage updates of the Runge-Kutta schemes (Sec. 3). */
pmg_status pmg_axpy(pmg_handle* h, int64_t n, double a, const double* x_dev, const double* y_dev, double* out_dev,
                    void* stream);

/* ---- learned warm start ---------------------------------------------------------------- */
/* A small periodic 1D convolutional network over the NX node columns of a tank predicts
 * the change of the pressure between consecutive solves of a time-stepping run; the
 * previous pressure plus that change is the initial guess of the next solve.  Not in the
 * paper (an addition of this library); FP32 parameters, activations and Adam moments.
 *
 * Input per column x (C = NZ + 3 + period channels): eta/s_eta, (eta - eta_prev)/s_deta,
 * eta_x, a one-hot of x mod period (period = the mesh order, so the network can tell
 * element-boundary columns from interior ones), p_prev(x, iz)/s_p for iz = 0..NZ-1, where
 * p_prev is the previous solve's pressure and eta_prev the surface it was solved on.
 * Layers: conv(taps) (C -> hidden), tanh,
 * conv(taps) (hidden -> hidden), tanh, conv(1) (hidden -> NZ); periodic in x (columns
 * wrap).  Output y (NZ x NX): guess = p_prev + s_dp * y, surface row left at p_prev.  The
 * last layer starts at zero, so an untrained network returns p_prev exactly.  Loss, with
 * e = y - (p - p_prev)/s_dp on the rows below the surface (the surface row is masked):
 * L = mean over nodes of e^2 + lam ((e(z+1) - e)^2 + (e(x+1) - e)^2), x periodic; lam
 * (default 0, see pmg_ws_set_roughness) weights rough errors, which cost the solve most.  The solve that follows always iterates to
 * its tolerance, so the network changes iteration counts, never the pressure returned.
 *
 * Parameters: one flat FP32 array [W1 (hidden, C, taps), b1 (hidden), W2 (hidden,
 * hidden, taps), b2 (hidden), W3 (NZ, hidden), b3 (NZ)], Glorot-uniform from `seed`
 * (SplitMix64), zero biases.  Device pointers below are float64 unless named float;
 * every call is asynchronous on `stream` unless it returns a host value.  Errors:
 * PMG_ERR_INVALID for NULL pointers, a batch size outside 1..max_batch or a shape that
 * does not match; PMG_ERR_OOM / PMG_ERR_CUDA from the runtime. */
typedef struct pmg_ws pmg_ws;
pmg_status pmg_ws_create(int n_cols, int col_len, int period, int hidden, int taps, int max_batch, uint64_t seed,
                         double s_eta, double s_deta, double s_p, double s_dp, pmg_ws** out);
pmg_status pmg_ws_destroy(pmg_ws* ws);
pmg_status pmg_ws_num_params(const pmg_ws* ws, int64_t* n);
/* Weight lam >= 0 of the first-difference terms of the training loss. */
pmg_status pmg_ws_set_roughness(pmg_ws* ws, double lam);
/* Host copies of the parameters out / in (n_params floats); setting resets Adam. */
pmg_status pmg_ws_get_params(pmg_ws* ws, float* host_out);
pmg_status pmg_ws_set_params(pmg_ws* ws, const float* host_in);
/* One sample's input (C x NX floats) and training target (NZ x NX floats). */
pmg_status pmg_ws_pack(pmg_ws* ws, const double* eta, const double* eta_prev, const double* etax,
                       const double* p_prev, float* in, void* stream);
pmg_status pmg_ws_target(pmg_ws* ws, const double* p, const double* p_prev, float* tgt, void* stream);
/* Forward pass of S samples (S x C x NX floats in, S x NZ x NX floats out). */
pmg_status pmg_ws_forward(pmg_ws* ws, const float* in, int S, float* out, void* stream);
/* x0 = p_prev + s_dp * net(input) (NX*NZ, z fastest). */
pmg_status pmg_ws_predict(pmg_ws* ws, const double* eta, const double* eta_prev, const double* etax,
                          const double* p_prev, double* x0, void* stream);
/* Loss of S samples and its gradient w.r.t. every parameter (n_params floats, device);
 * synchronises `stream` when loss_host is non-NULL. */
pmg_status pmg_ws_gradients(pmg_ws* ws, const float* in, const float* tgt, int S, float* grad, double* loss_host,
                            void* stream);
/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * loss of S samples. */
pmg_status pmg_ws_train_step(pmg_ws* ws, const float* in, const float* tgt, int S, float lr, double* loss_host,
                             void* stream);
/* Parameters to / from a file (header: magic, version, NX, NZ, period, hidden, taps). */
pmg_status pmg_ws_save(pmg_ws* ws, const char* path);
pmg_status pmg_ws_load(pmg_ws* ws, const char* path);

/* ---- batches of independent problems --------------------------------------------------- */
/* n independent tanks (each its own mesh, order and workspace), solved together.  Not in the
 * paper (it solves one tank at a time).  With the mixed precision (PMG_MIXED_FP32, outer
 * PMG_PCG or PMG_FCG, the default fast-diagonalisation smoother on flat levels, constant
 * depth, equal orders, double-float outer operator) and n <= 256, a batch solve is ONE CUDA
 * graph: every stage of the flexible-CG iteration -- each Schwarz sweep, level residual
 * and transfer of the V-cycle (levels aligned by their distance from the order-1 level),
 * the coarse solves, the outer operator, the Krylov vector updates -- is one launch whose
 * CTAs are the work items (element columns or nodes) of all problems, taken from a device
 * table; per-problem scalars, iteration counts, convergence flags and restarts on residual
 * drift live on the device, and a device-side while node runs until every problem is done.
 * Other options run each problem's own device-side loop on its own stream, concurrently.
 * opts apply to every problem; pmg_batch_create runs pmg_autotune on every problem (used by
 * the per-problem path). */
typedef struct pmg_batch pmg_batch;
pmg_status pmg_batch_create(int n, const pmg_mesh_desc* meshes, const pmg_opts* opts, pmg_batch** out);
pmg_status pmg_batch_destroy(pmg_batch* b);
/* The handle of problem i (owned by the batch): per-problem geometry and right-hand
 * sides are set through it with the single-problem calls. */
pmg_status pmg_batch_handle(pmg_batch* b, int i, pmg_handle** h);
/* Solve every problem: b[i], p_dirichlet[i], p_out[i] are device vectors of problem i
 * (x0 = 0).  infos (n entries) may be NULL.  Returns the first non-OK status (each
 * problem's own status is in its info).  Synchronises the caller's stream. */
pmg_status pmg_batch_solve(pmg_batch* b, const double* const* b_dev, const double* const* p_dirichlet_dev,
                           double* const* p_out_dev, pmg_solve_info* infos, void* stream);
/* How the batch solves: *batched = 1 for the single graph of batched launches, 0 for the
 * concurrent per-problem loops; *launches = kernel launches per iteration of the batched
 * graph (0 until its first solve has built it).  Any pointer may be NULL.  Host-side read;
 * no counterpart in the paper. */
pmg_status pmg_batch_info(const pmg_batch* b, int* batched, int* launches);
/* How later pmg_batch_solve calls run (no counterpart in the paper): path 0 (default) the
 * single graph of batched launches where the options allow it; 1 the same launches with
 * the iteration loop driven by the host (one host synchronisation per iteration: a kernel
 * profiler sees every launch; the same results); 2 each problem's own device-side loop on
 * its own stream, concurrently (as for options the batched launches do not cover).
 * PMG_ERR_INVALID for another value. */
pmg_status pmg_batch_set_path(pmg_batch* b, int path);

/* ---- autotuner ------------------------------------------------------------------------- */
/* Times the candidate launch configurations on every level of h (CUDA-event timing of
 * graph-captured launches) and keeps the fastest per kernel and shape for h; a later
 * candidate must be 3% faster to replace an earlier one.  Candidates: for the FP32 level
 * operator, slab CTAs of 64..512 threads, node-parallel CTAs of 64..256 and the tiled
 * shapes (constant-depth levels of equal orders up to 8), or only the family that
 * pmg_opts.flat_kernel forces; for the Schwarz sweep, the transfers and the
 * actual-geometry operators, CTA sizes of 64..512.  Where pmg_opts.fuse_residual = -1 it
 * also picks fused or split level residuals.  The paper has no counterpart (it fixes no
 * launch shapes).  The choices are also remembered per (kernel, order, rows, element
 * columns, forced family or arithmetic variant) for handles created later in the process,
 * and in the file named by PMG_TUNE_CACHE when set.  Synchronous; changes no results
 * (every candidate computes the same operator).  pmg_level_kernels reads the choices. */
pmg_status pmg_autotune(pmg_handle* h);

/* Bound of the handle's device-side waits (the z-split Schwarz sweep waits on an mbarrier
 * for its TMA slab copies): a wait that has not completed after `cycles` SM clock cycles
 * gives up, the CTA raises the handle's timeout flag, waits for its copies in flight and
 * leaves its part of the iterate unchanged.  cycles < 0 restores the default (2^31, about
 * one second); 0 gives up at once (how the tests exercise this path).  pmg_solve returns
 * PMG_ERR_TIMEOUT when the flag was raised since the previous pmg_solve (of any call on
 * the handle), and clears it.  The paper has no counterpart. */
pmg_status pmg_set_wait_limit(pmg_handle* h, int64_t cycles);

/* ---- allocation-free apply ------------------------------------------------------------ */
/* y = A_FF x on free nodes, y = x on the surface row -- the operator of pmg_apply on the
 * geometry eta (NX values), without a handle and without allocating device memory.  The
 * paper has no counterpart: this is for callers that cannot allocate (a host framework
 * that owns every device allocation, a fixed pool, a caller inside a stream capture).
 * The mesh must satisfy pmg_create's rules (pmg_level_sequence checks the same), with
 * order_z 0 or equal to order.  The geometry factors, sigma table and slab-edge exchange
 * buffers live in one static 4 MiB (4194304-byte) device array of the library (held by
 * every GPU that loads it, until exit).  A mesh needs
 *   256 + a(32 cells_x (order+1)) + a(8 NZ) + a(4 (cells_x+1)) + a(8 (cells_x+1) NZ) bytes,
 * NZ = cells_z order + 1, a(n) = n rounded up to a multiple of 256; larger meshes return
 * PMG_ERR_INVALID.  The first call on a device sets up (constant tables, the array's device
 * address via cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Asynchronous on the stream; x and y
 * are caller-owned device vectors of n = NX * NZ doubles.  The call reads nothing back, so
 * a depth d = eta + h that is not positive and finite somewhere (PMG_ERR_INVALID from the
 * handle path) shows in the output instead: every entry of y is NaN. */
pmg_status pmg_apply_noalloc(const pmg_mesh_desc* mesh, const double* eta_dev, const double* x_dev,
                             double* y_dev, void* stream);

/* ---- profiling ---------------------------------------------------------------------- */
/* Instrumentation of this library; no counterpart in the paper. */
/* Kernel classes for launch counting and device timing. */
enum {
  PMG_K_CURVED64 = 0,  /* actual-geometry operator, FP64 (apply / residual / dot)          */
  PMG_K_CURVED32 = 1,  /* actual-geometry operator, FP32                                    */
  PMG_K_LEVEL64 = 2,   /* flat level operator / residual, FP64                              */
  PMG_K_LEVEL32 = 3,   /* flat level operator / residual, FP32                              */
  PMG_K_SMOOTH64 = 4,  /* Schwarz smoother sweep, FP64                                      */
  PMG_K_SMOOTH32 = 5,  /* Schwarz smoother sweep, FP32                                      */
  PMG_K_TRANSFER = 6,  /* restriction and prolongation (both precisions)                    */
  PMG_K_COARSE = 7,    /* coarse solve (three launches per call)                            */
  PMG_K_VECTOR = 8,    /* Krylov vector kernels and reductions                              */
  PMG_K_SETUP = 9,     /* geometry factors and load vectors                                 */
  PMG_K_VCYCLE = 10,   /* fused coarse part of the FP32 V-cycle (one cooperative launch)    */
  PMG_K_COUNT = 11
};
/* Reset the per-class counters of h; timing != 0 also brackets every launch with CUDA
 * events on its stream (adds a small per-launch cost). */
pmg_status pmg_profile_reset(pmg_handle* h, int timing);
/* Per class since the last reset (host arrays of PMG_K_COUNT, any may be NULL): launch
 * counts, device milliseconds (zero unless timing was enabled), and the algorithmic bytes
 * and floating-point operations of those launches (the minimum DRAM traffic and work the
 * kernels' definitions imply; an FMA counts two).  Synchronises the device. */
pmg_status pmg_profile_read(pmg_handle* h, int64_t* launches, double* ms, double* bytes, double* flops);

/* Message of the last failing call on this thread ("" if none).  Error reporting of this
 * library; no counterpart in the paper. */
const char* pmg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PMG_H_ */
