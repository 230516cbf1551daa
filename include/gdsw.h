/*
 * gdsw.h -- C ABI of libgdsw.so: monolithic multilevel GDSW overlapping Schwarz
 * preconditioner and flexible GMRES for Q2/Q1 Carreau Stokes saddle-point systems,
 * computed on one GB300 (sm_103a) GPU.
 *
 * Method (arXiv 2606.01433):
 *   - Section 2, saddle-point equation: A_cal = [[A, B^T], [B, 0]] from the weak form
 *     mu int grad u : grad v - int div v p (gradient form) or, Section 3,
 *     int 2 nu(u_k) D(u):D(v) - int div v p (symmetric form, Carreau nu).
 *   - Section 2.1: overlapping restrictions R_i, local saddle-point matrices
 *     A_i = R_i A R_i^T, interface entities, coarse basis Phi by saddle-point extension,
 *     A_0 = Phi^T A Phi, B = Phi A_0^{-1} Phi^T + sum_i R_i^T A_i^{-1} R_i.
 *   - Section 2.2: multilevel recursion and the four-level preconditioner equation; only
 *     the coarsest A_0^(L) is solved directly.
 *   - Section 3: restarted FGMRES preconditioned by the multilevel operator.
 *
 * Conventions shared by every call:
 *   - Mesh: nx*ny*nz axis-aligned cubes of edge h; element (ex,ey,ez) has index
 *     ex + nx*(ey + ny*ez); Q2 node (i,j,k), 0 <= i <= 2nx, at origin + (h/2)(i,j,k), has
 *     index i + (2nx+1)*(j + (2ny+1)*k).  Q1 (pressure) nodes are the Q2 nodes with all
 *     indices even that belong to a fluid element.
 *   - Free-dof vector order: free velocity nodes (fluid nodes whose tag is not
 *     GDSW_TAG_WALL / GDSW_TAG_INFLOW) in increasing node index, three interleaved
 *     components each, then the pressure nodes in increasing node index.  n = 3 n_vnodes +
 *     n_pnodes.
 *   - Vectors passed to gdsw_apply / gdsw_spmv / gdsw_solve / gdsw_rhs_lift are DEVICE
 *     pointers to contiguous float64 arrays of length n, owned by the caller.  Calls are
 *     ordered on the context's stream; apply/spmv/rhs_lift return without synchronising;
 *     gdsw_solve returns after the final status is known.
 *   - Host arrays passed to gdsw_setup are read during the call only.
 *   - The context owns every factor, basis and workspace; gdsw_destroy frees them.
 *   - Every call returns GDSW_OK or an error code; gdsw_last_error gives the message.
 *     No exception crosses the ABI.  A context whose call returned GDSW_ERR_CUDA should be
 *     destroyed.
 */
#ifndef GDSW_H
#define GDSW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum gdsw_status {
  GDSW_OK = 0,
  GDSW_ERR_INVALID_ARG = 1,
  GDSW_ERR_OOM = 2,
  GDSW_ERR_SINGULAR = 3,      /* a pivot of a local / coarse factorisation vanished */
  GDSW_ERR_NOT_CONVERGED = 4, /* FGMRES hit max_it; x holds the last iterate */
  GDSW_ERR_NAN = 5,           /* non-finite residual */
  GDSW_ERR_TIMEOUT = 6,       /* a bounded device wait expired */
  GDSW_ERR_CUDA = 7
};

enum gdsw_tag { GDSW_TAG_INTERIOR = 0, GDSW_TAG_WALL = 1, GDSW_TAG_INFLOW = 2, GDSW_TAG_OUTFLOW = 3 };
enum gdsw_form { GDSW_FORM_GRADIENT = 0, GDSW_FORM_SYMMETRIC = 1 };
enum gdsw_precision { GDSW_FP64 = 0, GDSW_FP32 = 1, GDSW_BF16 = 2 };
/* Engine of the FP32 set-up GEMMs (local factorisation, coarse basis): the tensor cores with
 * the 3xTF32 split (AUTO, the default, for tasks of at least 96 x 96 outputs), or SIMT FMA. */
enum gdsw_gemm_engine { GDSW_GEMM_AUTO = 0, GDSW_GEMM_SIMT = 1, GDSW_GEMM_TENSOR = 2 };
enum gdsw_weighting { GDSW_WEIGHT_POU = 0, GDSW_WEIGHT_PLAIN = 1 };
/* Pressure element: continuous Q1 (Taylor-Hood, one dof per even-index node) or the paper's
 * discontinuous P1 (Section 2: four dofs per fluid element -- the coefficients of 1, xi, eta,
 * zeta in the element's reference coordinates [-1, 1]^3 -- numbered 4 f + k after the velocity
 * dofs, f the fluid element's rank in element order). */
enum gdsw_pressure { GDSW_PRESSURE_Q1 = 0, GDSW_PRESSURE_P1DISC = 1 };

typedef struct gdsw_ctx gdsw_ctx;

/* Voxel mesh and boundary data (Section 3 model problem: inflow, outflow, no-slip). */
typedef struct {
  int32_t nx, ny, nz;
  double h;
  double origin[3];
  const uint8_t* mask;   /* host, nx*ny*nz; 1 = fluid element */
  const uint8_t* tags;   /* host, (2nx+1)(2ny+1)(2nz+1) node tags (enum gdsw_tag) */
  const double* g;       /* host, 3 per node: Dirichlet datum (read where tag is WALL/INFLOW) */
  int32_t pressure;      /* a gdsw_pressure value; 0, the zero-initialised default, is Q1.
                            P1-disc coarse spaces hold one pressure column per part on every
                            level; P1-disc grids take no multigrid hierarchy; any other value
                            is GDSW_ERR_INVALID_ARG. */
} gdsw_mesh;

/* Viscosity (Section 2: constant mu; Section 3: Carreau law
 * nu = nu_inf + (nu0 - nu_inf)(1 + (lambda gamma_dot)^2)^((n-1)/2),
 * gamma_dot = sqrt(2 D(u_k):D(u_k)) at every Gauss point of the frozen velocity u_k). */
typedef struct {
  int32_t form;          /* enum gdsw_form */
  double nu0, nu_inf, lambda, n;
  const double* uk;      /* host, 3 per node, or NULL: constant nu0 */
} gdsw_viscosity;

/* Partition (Section 2.1 nonoverlapping subdomains; Section 2.2 coarser parts). */
typedef struct {
  const int32_t* elem_part;   /* host, nx*ny*nz: subdomain of each fluid element (>= 0) */
  int32_t n_groups;           /* levels - 2 grouping arrays */
  const int32_t* groups[2];   /* groups[l][p] = level-(l+2) part of level-(l+1) part p */
  int32_t group_len[2];       /* entries in groups[l] (= number of level-(l+1) parts) */
} gdsw_partition;

typedef struct {
  int32_t levels;        /* L in {2,3,4}: L-1 Schwarz levels, direct solve of A_0^(L); 1: operator only */
  int32_t overlap;       /* element layers of overlap on level 1 (the paper uses 1) */
  int32_t rotations;     /* 1: add the rigid rotations about each entity's centroid to the
                            level-1 coarse space (the null-space enrichment Section 2.1 leaves
                            out; two levels only); 0: translations and pressure constants */
} gdsw_levels;

typedef struct {
  int32_t weighting;        /* enum gdsw_weighting */
  int32_t precision[3];     /* storage precision of the local factors on Schwarz levels 1..3 */
  int32_t phi_precision;    /* storage precision of the level-1 coarse basis */
  int32_t restart;          /* FGMRES restart length m */
  int32_t max_it;
  double tol;               /* relative residual ||b - A x|| / ||b|| */
  int32_t slab_elems;       /* level-1 factor slab thickness in elements; 0 = one dense block */
  int32_t use_graph;        /* capture the preconditioner apply in a CUDA graph */
  void* stream;             /* cudaStream_t for all work of this context (NULL = default) */
} gdsw_options;

typedef struct {
  int32_t iterations;
  int32_t status;           /* enum gdsw_status of the solve */
  double relres;            /* true ||b - A x|| / ||b|| in FP64 */
  double est_relres;        /* the Krylov estimate at exit */
  double time_ms;           /* device time of the whole solve */
  double apply_ms;          /* summed device time of preconditioner applies */
  double spmv_ms;
  double arnoldi_ms;
} gdsw_solve_info;

typedef struct {
  int64_t n, n_u, n_p, n_elems, n_nodes;
  int32_t levels;
  int64_t n_coarse[4];      /* n_coarse[l] = size of A_0^(l+2) (l = 0..L-2) */
  int32_t n_parts[3];       /* parts on Schwarz levels 1..L-1 */
  int64_t local_dofs[3];    /* sum of overlapping local sizes per Schwarz level */
  int64_t factor_entries[3];/* stored factor entries per Schwarz level */
  int64_t max_local[3];     /* largest local problem per Schwarz level */
  int32_t max_slabs;        /* level-1 block-tridiagonal depth */
  int64_t nnzb_A, nnz_B;    /* 3x3 velocity blocks; pressure-velocity 1x3 entries */
  int64_t phi_entries;      /* stored level-1 Phi_I entries */
  int64_t device_bytes;     /* bytes the context holds on the device */
  double setup_ms[6];       /* host symbolic, viscosity+assembly, level-1 factors, Phi+A0,
                               coarse levels, total */
  int32_t tile_rows[3];     /* rows per forward GEMV tile chosen by the set-up autotuner */
  int32_t persistent[3];    /* 1: local solve as one persistent launch (autotuner's choice) */
  double tuned_ms[3];       /* the chosen configuration's local-solve time (0: not tuned) */
} gdsw_sizes_info;

/* Per-call kernel timing (CUDA events on the context stream) and algorithmic bytes.  The
 * gather, local, scatter, restrict and prolong groups hold level-1 work only; everything on
 * the coarser levels (their gathers, local solves, scatters and transfers, and the coarsest
 * direct solve) is the coarse group. */
typedef struct {
  int32_t enabled;
  int64_t calls[12];
  double ms[12];
  double bytes[12];         /* algorithmic bytes moved per call, summed */
} gdsw_profile;

enum gdsw_kernel_group {
  GDSW_K_SPMV = 0, GDSW_K_GATHER = 1, GDSW_K_LOCAL = 2, GDSW_K_SCATTER = 3,
  GDSW_K_RESTRICT = 4, GDSW_K_COARSE = 5, GDSW_K_PROLONG = 6, GDSW_K_ARNOLDI = 7,
  GDSW_K_APPLY = 8, GDSW_K_ASSEMBLY = 9, GDSW_K_VISCOSITY = 10, GDSW_K_OTHER = 11
};

/* Build everything: host symbolic setup (dofs, patterns, overlap, entities, orderings),
 * then on the device the Carreau viscosity, the assembly of A_cal, the local factors of
 * every Schwarz level, the coarse bases and coarse operators, and the direct inverse of
 * the coarsest operator.  Returns GDSW_ERR_SINGULAR if a factorisation pivot vanishes. */
int gdsw_setup(const gdsw_mesh* mesh, const gdsw_viscosity* visc, const gdsw_partition* part,
               const gdsw_levels* levels, const gdsw_options* opt, gdsw_ctx** out);

/* Host-only analysis with the same arguments: dof numbering, overlapping subdomains,
 * entities and coarse sizes of every level (Section 2.1 / 2.2 index sets), plus an
 * estimate of the device memory gdsw_setup would take (gdsw_sizes_info.device_bytes).
 * Touches no GPU.  The returned context answers gdsw_sizes, gdsw_level_dofs and
 * gdsw_level_entities; every device call on it returns GDSW_ERR_INVALID_ARG. */
int gdsw_analyze(const gdsw_mesh* mesh, const gdsw_viscosity* visc, const gdsw_partition* part,
                 const gdsw_levels* levels, const gdsw_options* opt, gdsw_ctx** out);

void gdsw_destroy(gdsw_ctx* ctx);
const char* gdsw_last_error(const gdsw_ctx* ctx);
int gdsw_sizes(const gdsw_ctx* ctx, gdsw_sizes_info* info);

/* b = -A_(free, Dirichlet) g (Section 2: inhomogeneous Dirichlet datum moved to the right
 * side); b is a device vector of length n. */
int gdsw_rhs_lift(gdsw_ctx* ctx, double* b);

/* y = A_cal x (Section 2 saddle-point equation), FP64. */
int gdsw_spmv(gdsw_ctx* ctx, const double* x, double* y);

/* z = B r: the multilevel GDSW preconditioner (Section 2.2 four-level equation and its
 * two/three-level forms), with the precisions chosen at setup. */
int gdsw_apply(gdsw_ctx* ctx, const double* r, double* z);

/* Restarted FGMRES (Section 3) for A_cal x = b; x holds the initial guess on entry. */
int gdsw_solve(gdsw_ctx* ctx, const double* b, double* x, gdsw_solve_info* info);

/* The same solve with HOST buffers: the copies to and from the device are part of the call. */
int gdsw_solve_host(gdsw_ctx* ctx, const double* b_host, double* x_host, gdsw_solve_info* info);

/* Re-evaluate the Carreau viscosity from a new frozen velocity u_k (host array, 3 per node,
 * or NULL to keep the current one) and re-assemble A_cal in place (a Picard step with a
 * frozen preconditioner). */
int gdsw_reassemble(gdsw_ctx* ctx, const double* uk_host);
/* Picard update of the nonlinear Carreau iteration (Section 3, the Picard half of its
 * alternating Picard-Newton loop): the frozen velocity u_k becomes the velocity of the
 * solution x (device FP64, free dofs in gdsw_solve order) at the free nodes and the Dirichlet
 * data g at the others.  The next gdsw_reassemble(ctx, NULL) then evaluates nu(u_k) and
 * re-assembles; the preconditioner keeps its factors (a frozen-preconditioner Picard step; a
 * new context refactors).  Newton terms are not provided: they make A non-symmetric.
 * Asynchronous on the context stream. */
int gdsw_picard_update(gdsw_ctx* ctx, const double* x);

/* r = b - A x with the current operator (device FP64 vectors). */
int gdsw_residual(gdsw_ctx* ctx, const double* b, const double* x, double* r);

/* One Newton step of Section 3's alternating Picard-Newton iteration, from the state x (device
 * FP64, free dofs; u_k must be its velocity, as after gdsw_picard_update(ctx, x)): evaluate
 * nu(u_k), assemble the Picard operator A(nu(u_k)) and form the nonlinear residual
 * R = b(nu(u_k)) - A(nu(u_k)) x, add the Newton term of the Carreau law,
 * int 4 nu'(gamma_dot)/gamma_dot (D(u_k):D(w)) (D(u_k):D(v)) -- symmetric, since the Carreau
 * problem minimises a convex energy, so the symmetric block-LDL^T factors of the frozen
 * preconditioner still apply -- solve J delta = R by FGMRES from zero, then x += delta and
 * u_{k+1} = x's velocity with the Dirichlet data.  Afterwards the context's operator is the
 * Jacobian; gdsw_reassemble restores the Picard operator.  Needs the symmetric form and a
 * velocity (GDSW_ERR_INVALID_ARG otherwise).  info: the linear solve's record.  Synchronous. */
int gdsw_newton_step(gdsw_ctx* ctx, double* x, gdsw_solve_info* info);

/* ---- geometric multigrid with the multilevel GDSW method as its coarse solver ----
 * Section 3 of the paper also uses the Schwarz method as the coarse-grid solver of a
 * geometric multigrid method: FGMRES preconditioned by it solves the coarsest problem to a
 * relative residual of 1e-1.  Here the grids are contexts of nested voxel meshes (each twice
 * as fine as the next, same fluid region), finest first, all on one stream: the fine grids
 * set up with levels = 1 (operator only: assembly, SpMV, lifting), the coarsest with its
 * multilevel GDSW preconditioner, whose FGMRES tolerance (gdsw_options.tol) is the
 * coarse-solve tolerance.  gdsw_mg_create builds, on every fine grid, the element-Vanka
 * patches (the free dofs of an element's 27 Q2 and 8 Q1 nodes; explicit inverses of the
 * principal submatrices of the assembled operator, inverted in FP64 and stored in the
 * smoother precision) and the transfer to the next coarser grid (nodal interpolation P of
 * Q2 velocity and Q1 pressure, zero at coarse Dirichlet nodes; R = P^T), and attaches the
 * V-cycle as the preconditioner of the finest context: gdsw_solve on grids[0] then runs FP64
 * FGMRES preconditioned by V-cycles.  A smoothing step is a multiplicative sweep over the
 * eight element colours (parity of the voxel indices): r = b - A z, then every patch e of the
 * colour adds omega A_e^{-1} r_e to z; FP64 smoothing forms r with the FP64 SpMV, FP32
 * smoothing only on the rows the colour's patches touch, with FP32 operator values copied
 * when the multigrid is created (re-create it after re-assembling a grid's operator).  The multigrid object does not own the grid
 * contexts; destroy it before them.  Errors as for the other calls; a failed create leaves
 * its reason in gdsw_mg_last_error(NULL). */
typedef struct gdsw_mg gdsw_mg;
typedef struct gdsw_mg_options {
  double omega;                 /* Vanka damping (1 = undamped) */
  int32_t pre, post;            /* smoothing steps before / after the coarse correction */
  int32_t smoother_precision;   /* GDSW_FP32 (patch inverses and products in FP32) or GDSW_FP64 */
  int32_t symmetric;            /* 1: post-smoothing sweeps the colours in reverse order */
} gdsw_mg_options;
int gdsw_mg_create(gdsw_ctx* const* grids, int32_t ngrids, const gdsw_mg_options* opt, gdsw_mg** out);
void gdsw_mg_destroy(gdsw_mg* mg);
const char* gdsw_mg_last_error(const gdsw_mg* mg);
/* z = V r: one V-cycle from a zero initial guess (device FP64 vectors of the finest grid). */
int gdsw_mg_vcycle(gdsw_mg* mg, const double* r, double* z);
/* steps smoothing steps on fine grid `grid` (0 = finest), x updated in place. */
int gdsw_mg_smooth(gdsw_mg* mg, int32_t grid, const double* b, double* x, int32_t steps);
/* zf += P xc from grid+1 to grid; rc = R rf = P^T rf from grid to grid+1. */
int gdsw_mg_prolong(gdsw_mg* mg, int32_t grid, const double* xc, double* zf);
int gdsw_mg_restrict(gdsw_mg* mg, int32_t grid, const double* rf, double* rc);
/* V-cycles run, coarse solves and their total FGMRES iterations since creation. */
int gdsw_mg_stats(const gdsw_mg* mg, int64_t* cycles, int64_t* coarse_solves, int64_t* coarse_iterations);

/* ---- component access for tests and profiling (same arithmetic as the apply) ---- */

/* Level l (0-based Schwarz level) local branch only: z = sum_i R_i^T D_i A_i^{-1} R_i r
 * (D_i = I for plain weighting).  r, z: device FP64 vectors of that level's size. */
int gdsw_apply_local(gdsw_ctx* ctx, int32_t level, const double* r, double* z);
/* The same result as gdsw_apply_local, computed without allocating any memory: for callers
 * that must not call cudaMalloc/cudaFree while they run -- a process that has handed every
 * free byte of the device to its own memory pool, or a latency-critical loop that cannot
 * afford the device-wide synchronisation a cudaFree implies.  The paper has no counterpart;
 * this is an interface variant of the level-l local branch.
 *   - Scratch: a fixed 4 MiB (4,194,304-byte) 256-byte-aligned array in the library's device
 *     memory, held by every GPU that loads the library until the process exits.  The level's
 *     concatenated local vectors and the partial sums of its packed symmetric blocks
 *     ((2 x local dofs + partials) x 8 bytes for FP64 factors, x 4 for FP32/BF16) must fit;
 *     larger levels get GDSW_ERR_INVALID_ARG with the size in gdsw_last_error.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current); make that first call before any stream capture.  The
 *     device current at the call must be the one the context was set up on (else
 *     GDSW_ERR_INVALID_ARG).  The address is kept until the process exits: no call may
 *     follow a cudaDeviceReset of that device.
 *   - Every call on a device shares the one array and leaves the last call's values in it;
 *     nothing has to start at zero (each entry read is written earlier in the same call).
 *     Calls that overlap on the GPU (other streams, other threads, other contexts) race.
 *   - r, z: device FP64 vectors of the level's size, as for gdsw_apply_local; the call is
 *     asynchronous on the context's stream. */
int gdsw_apply_local_noalloc(gdsw_ctx* ctx, int32_t level, const double* r, double* z);

/* r0 = Phi^T r towards level l+1 (device vectors). */
int gdsw_restrict(gdsw_ctx* ctx, int32_t level, const double* r, double* r0);
/* z += Phi x0 (device vectors). */
int gdsw_prolong(gdsw_ctx* ctx, int32_t level, const double* x0, double* z);
/* Copy the coarse operator A_0^(l+2) (dense, row-major FP64, n_coarse[l]^2) to host. */
int gdsw_coarse_matrix(gdsw_ctx* ctx, int32_t l, double* host);
/* Copy the assembled operator to host as CSR on free dofs: row_ptr (n+1), col (nnz),
 * val (nnz); pass NULL pointers to query nnz through *nnz. */
int gdsw_matrix_csr(gdsw_ctx* ctx, int64_t* row_ptr, int32_t* col, double* val, int64_t* nnz);
/* Copy the Gauss-point viscosity nu[e][27] (fluid elements in increasing index) to host. */
int gdsw_viscosity_values(gdsw_ctx* ctx, double* host);
/* Level-l overlapping sets: dof lists of every subdomain concatenated (global numbering of
 * that level, sorted per subdomain) and their offsets (n_parts + 1). */
int gdsw_level_dofs(gdsw_ctx* ctx, int32_t level, int64_t* offsets, int32_t* dofs);
/* Coarse-space columns: for level l, the number of entities and their modes. */
int gdsw_level_entities(gdsw_ctx* ctx, int32_t level, int32_t* n_entities);

/* Number of CUDA kernels this library has launched in this process (all contexts). */
int64_t gdsw_kernel_launches(void);

/* One FP32 GEMM task of the set-up: C = alpha op(A) op(B) + beta C, row-major device
 * matrices (op(A) = A^T when trans_a, op(B) = B^T when trans_b; op(A) is M x K, op(B) K x N). */
typedef struct gdsw_gemm_task {
  const float* a;
  const float* b;
  float* c;
  int32_t M, N, K, lda, ldb, ldc, trans_a, trans_b;
  double alpha, beta;
} gdsw_gemm_task;

/* The batched FP32 GEMM of the set-up (the dense contractions of the local block-LDL^T
 * factorisation of Section 2.1's A_i and of the coarse basis Phi_I = -A_II^{-1} A_IGamma
 * Phi_Gamma): engine GDSW_GEMM_TENSOR runs every task on the tensor cores (tcgen05 kind::tf32,
 * TMA-staged, 3xTF32 split, FP32 accumulation; needs M, N, K >= 1), GDSW_GEMM_SIMT on the
 * SIMT kernels, GDSW_GEMM_AUTO as the set-up does.  Tasks must not overlap in C.  Synchronous
 * (on the legacy default stream); GDSW_ERR_TIMEOUT if a pipeline wait of the tensor-core
 * kernel gave up, GDSW_ERR_INVALID_ARG for a bad task. */
int gdsw_gemm_f32(const gdsw_gemm_task* tasks, int32_t ntasks, int32_t engine);

/* Default engine of the FP32 set-up GEMMs for contexts set up afterwards (process-wide). */
int gdsw_set_gemm_engine(int32_t engine);

/* Overlapped launch chain of the batched GEMV sweeps (process-wide, default on): each launch
 * of a local solve is made with programmatic dependent launch, so that its CTAs can become
 * resident and prefetch their factor rows while the previous launch drains; they wait for the
 * previous launch's completion before reading any vector, so results are bitwise the same with
 * the chain on (1) or off (0).  Returns GDSW_OK, or GDSW_ERR_INVALID_ARG for another value. */
int gdsw_set_launch_overlap(int32_t on);

/* FMA throughput of the current device in TFLOP/s (precision GDSW_FP64 or GDSW_FP32): one
 * launch of independent fused multiply-add chains (8 per thread, 8 CTAs of 256 threads per
 * SM), timed with CUDA events after a warm-up launch.  It is the arithmetic roofline of the
 * FP64 operator kernels (SpMV, assembly, Arnoldi), which GB300's narrow FP64 pipe bounds
 * rather than memory.  Synchronous; allocates a small output buffer with cudaMalloc.
 * Returns GDSW_ERR_INVALID_ARG for another precision or a NULL pointer. */
int gdsw_probe_fma(int32_t precision, double* tflops);

/* Algorithmic bytes of one launch of the level-l local-solve sweeps: direction 0 = forward
 * launches (k = 0 .. K-1), 1 = backward launches (k = 0 .. K-2), in launch order, 2 = the
 * partial-sum reduction of the packed symmetric blocks (k = 0; 0 bytes when none).  Used to
 * put the DRAM traffic of a profiled launch beside the bytes the method must move. */
int gdsw_plan_bytes(const gdsw_ctx* ctx, int32_t level, int32_t direction, int32_t k, double* bytes);

/* How the local solves of every level run (the arithmetic, and so the result, is the same
 * bit for bit either way):
 *   persistent = 0: one launch per slab step, forward then backward (Section 2.1
 *     A_i^{-1} applied as block-LDL^T sweeps);
 *   persistent = 1: one persistent launch per level and apply; CTAs take the tiles of all
 *     slab steps from a work list in dependency order and wait (at most 1 s per wait, else
 *     gdsw_solve returns GDSW_ERR_TIMEOUT) until the tiles they read from are written.
 * ctas_per_sm: resident CTAs per SM of the persistent launch (0 = as many as fit); fewer
 * leave room for the coarse branch that runs concurrently on a second stream.
 * tile_rows: rows per forward GEMV tile, 32, 64 or 128 (0 = keep).  gdsw_setup chooses the
 * level-1 mode and tile rows by timing applies (gdsw_sizes reports the choice); this call
 * overrides it for every level.  Must not be called while the context has work in flight or
 * inside a stream capture; a context whose apply is captured in a CUDA graph (use_graph)
 * keeps its mode (GDSW_ERR_INVALID_ARG). */
int gdsw_set_local_sweep(gdsw_ctx* ctx, int32_t persistent, int32_t ctas_per_sm, int32_t tile_rows);

/* Failure-path self-test of the persistent sweep's bounded waits: runs the level-1 sweep once
 * with one dependency raised beyond what its producers signal, so that wait can never be met.
 * The wait gives up after its 1 s limit, every CTA returns, and the call reports
 * GDSW_ERR_TIMEOUT (GDSW_ERR_CUDA if no timeout was seen).  The GPU is never left waiting;
 * the context stays usable (the next apply starts from fresh counters and gathers anew). */
int gdsw_sweep_wait_selftest(gdsw_ctx* ctx);

int gdsw_profile_enable(gdsw_ctx* ctx, int32_t on);
int gdsw_profile_read(gdsw_ctx* ctx, gdsw_profile* prof);
int gdsw_profile_reset(gdsw_ctx* ctx);

/* ---- serving: continuous batching of independent Stokes solves ------------------------ *
 * A server owns one GPU, a device-memory budget and a number of slots (worker threads, each
 * with its own CUDA stream).  Submitted requests are analysed on the host (gdsw_analyze's
 * symbolic set-up gives the exact sizes and a device-memory estimate), admitted as soon as a
 * slot is free and the estimate fits in the remaining budget, then set up, solved and
 * released on their slot's stream, so the work of several requests overlaps on the device
 * while later requests keep arriving.  Requests that can never fit fail with GDSW_ERR_OOM.
 * Every result is computed by the same deterministic kernels as gdsw_solve, so a request
 * gives the same x whether it runs alone or in a mix. */
typedef struct gdsw_server gdsw_server;

typedef struct {
  gdsw_mesh mesh;           /* host arrays are copied at submit */
  gdsw_viscosity visc;
  gdsw_partition part;
  gdsw_levels levels;
  gdsw_options opt;         /* opt.stream is ignored: the slot's stream is used */
  const double* rhs;        /* host right-hand side of length x_len, or NULL: lifted Dirichlet data */
  double* x;                /* host result buffer of x_len doubles; must stay valid until completion */
  int64_t x_len;            /* must equal the problem's n (gdsw_analyze gives it) */
} gdsw_request;

enum gdsw_request_state {
  GDSW_REQ_QUEUED = 0, GDSW_REQ_ANALYSING = 1, GDSW_REQ_WAITING = 2, GDSW_REQ_RUNNING = 3,
  GDSW_REQ_DONE = 4, GDSW_REQ_FAILED = 5
};

typedef struct {
  int32_t state;            /* enum gdsw_request_state */
  int32_t status;           /* gdsw_status of the request once done or failed */
  int32_t iterations;
  int32_t slot;
  int64_t n;
  int64_t est_bytes;        /* admission estimate */
  double relres;
  double queue_ms;          /* submit -> memory reserved */
  double setup_ms;          /* device set-up */
  double solve_ms;          /* right-hand side, FGMRES and the copy back */
  double latency_ms;        /* submit -> result in the caller's buffer */
} gdsw_request_status;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t budget_bytes, used_bytes, peak_used_bytes;
  int32_t running, peak_running;
} gdsw_server_stats;

/* device: CUDA ordinal; mem_budget_bytes: device memory the server may reserve for requests;
 * max_slots: requests in flight at once (1..64). */
int gdsw_server_create(int32_t device, int64_t mem_budget_bytes, int32_t max_slots, gdsw_server** out);
/* Queue a request; *ticket identifies it.  Host inputs are copied before the call returns. */
int gdsw_server_submit(gdsw_server* srv, const gdsw_request* req, int64_t* ticket);
/* Non-blocking status of a ticket. */
int gdsw_server_poll(gdsw_server* srv, int64_t ticket, gdsw_request_status* st);
/* Block until the ticket is done or failed. */
int gdsw_server_wait(gdsw_server* srv, int64_t ticket, gdsw_request_status* st);
int gdsw_server_stats_read(gdsw_server* srv, gdsw_server_stats* st);
/* Finish every queued request, stop the workers and free the server. */
int gdsw_server_destroy(gdsw_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* GDSW_H */
