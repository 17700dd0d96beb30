/*
 * sem.h -- C ABI of the GB300 (sm_103a) spectral-element pressure-Poisson
 * library (libsem_gb300.so).
 *
 * The operations follow the paper "Experience and Analysis of Scalable
 * High-Fidelity Computational Fluid Dynamics on Modular Supercomputing
 * Architectures" (Karp et al., arXiv 2405.05640), section 3.1 ("Neko"): the
 * domain is split into E hexahedral elements carrying an order-N Lagrange
 * basis on the Gauss-Lobatto-Legendre (GLL) points; every operator except
 * the gather-scatter acts element by element (matrix-free); the gather-
 * scatter sums the copies of nodes shared between elements; a preconditioned
 * Krylov method solves Ax = b each time step.  Section 4.2 notes that the
 * solver is memory bound and that the gather-scatter is the communication
 * kernel.  Formulas are the textbook SEM ones the paper cites (Deville,
 * Fischer & Mund 2002).
 *
 * Conventions (all entry points):
 *  - Every device pointer is owned by the caller.  The library allocates no
 *    device memory: sem_mesh_create places its arrays in a caller-supplied
 *    device workspace, sem_pcg_solve uses a caller-supplied scratch buffer.
 *    Host pointers are read during the call only.
 *  - Fields are element-local ("E-layout"): u[e][k][j][i], i fastest,
 *    E * (N+1)^3 contiguous values, element e = ex + nx*(ey + ny*ez).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    are stream-ordered and asynchronous unless stated otherwise.
 *  - Return value: SEM_OK or a negative SEM_ERR_* code; no call aborts the
 *    process.  sem_last_error() gives a message for the calling thread.
 *  - Thread safety: calls on distinct meshes may run concurrently from
 *    different host threads.
 */
#ifndef SEM_GB300_H
#define SEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_OK 0
#define SEM_ERR_INVALID_ARG (-1)
#define SEM_ERR_CUDA (-2)
#define SEM_ERR_MESH (-3)          /* det J <= 0 somewhere */
#define SEM_ERR_WORKSPACE (-4)     /* workspace / scratch too small or misaligned */
#define SEM_ERR_NAN (-5)           /* NaN or Inf in the right-hand side */
#define SEM_ERR_NOT_CONVERGED (-6) /* max_iter reached; x and stats still filled */
#define SEM_ERR_TIMEOUT (-7)       /* a bounded device wait gave up */
#define SEM_ERR_UNSUPPORTED (-8)   /* order N or option not built */

#define SEM_MAX_ORDER 11           /* 1 <= N <= SEM_MAX_ORDER */

/* Data types of field arguments. */
#define SEM_F64 0
#define SEM_F32 1
#define SEM_F64_PAIR 2             /* FP64 fields, operator evaluated in double-float
                                      (FP32-pair, ~48-bit) arithmetic: an
                                      approximation of the FP64 operator, not
                                      FP64 arithmetic (see sem_ax) */

/* Extra precision copies of the geometric factors that sem_mesh_create
 * builds (bitmask; FP64 factors are always built). */
#define SEM_GEOM_F32 1             /* FP32 factors for the FP32 operator */
#define SEM_GEOM_RX 2              /* inverse Jacobian dr_a/dx_m (9 per point, FP64):
                                      needed by sem_gradient, sem_advect,
                                      sem_weak_div and the sem_ns_* stepper */
#define SEM_GEOM_PAIR 4            /* FP32-pair (hi, lo) factors, 48 bytes per point,
                                      for sem_ax with SEM_F64_PAIR */
#define SEM_GEOM_AFFINE 8          /* every element is an axis-aligned box (checked;
                                      SEM_ERR_MESH otherwise): the FP32 operator
                                      (sem_ax SEM_F32, the mixed solver's inner loop)
                                      then forms G = rho_i rho_j rho_k (a, b, c)_e
                                      from 3 scalars per element instead of reading
                                      6 factors per point (20 instead of 44 bytes
                                      per point in the fused CG operator); needs
                                      SEM_GEOM_F32 */
#define SEM_GEOM_BF16 16           /* BF16 copy of the six factors (12 bytes per point):
                                      the FP32 operator (sem_ax SEM_F32, the mixed
                                      solver's inner loop) reads it instead of the
                                      FP32 factors (32 instead of 44 bytes per point
                                      in the fused CG operator; FP32 arithmetic, the
                                      factors rounded to 8 bits); needs SEM_GEOM_F32 */

typedef struct sem_mesh sem_mesh;  /* opaque; freed by sem_mesh_destroy */

/* A box of nel[0] x nel[1] x nel[2] hexahedra.  Topology: local point
 * (e; i,j,k) of element (ex,ey,ez) is the global node
 * (ex*N+i, ey*N+j, ez*N+k), wrapped on periodic axes.  Geometry: the
 * trilinear map of the 8 vertices of each element (any hexahedra with a
 * positive Jacobian; the box only fixes which nodes are shared). */
typedef struct {
    int N;                 /* polynomial order, 1..SEM_MAX_ORDER */
    int nel[3];            /* elements per axis, each >= 1 */
    int periodic[3];       /* nonzero = periodic axis */
    int dirichlet_faces;   /* bit 2a: low face of axis a, bit 2a+1: high face;
                              ignored on periodic axes */
    const double *vertices;/* HOST array [E][8][3], vertex v = vx+2vy+4vz */
    int geom_flags;        /* SEM_GEOM_* bitmask */
} sem_mesh_desc;

typedef struct {
    int N;
    int64_t E;             /* number of elements */
    int64_t nloc;          /* E * (N+1)^3 element-local points */
    int64_t nglob;         /* unique global nodes (including Dirichlet nodes) */
    int64_t n_paper;       /* E * N^3, the paper's DOF count (Table 1) */
    int64_t n_shared_groups;  /* gather-scatter groups (shared or masked nodes) */
    int64_t n_shared_points;  /* local points in those groups */
    size_t workspace_bytes;   /* bytes of the mesh workspace in use */
} sem_mesh_info;

/* Library version string and message for the calling thread's last error. */
const char *sem_version(void);
const char *sem_last_error(void);
const char *sem_status_string(int status);

/* Bytes of device workspace sem_mesh_create needs for `desc` (0 on invalid
 * arguments).  Builds the host-side connectivity to count shared nodes. */
size_t sem_mesh_workspace_bytes(const sem_mesh_desc *desc);

/* Build a mesh: copy the vertices to the device, compute the geometric
 * factors G (six per point: rr, ss, tt, rs, rt, st, each
 * rho_i rho_j rho_k detJ sum_m dr_a/dx_m dr_b/dx_m), the diagonal mass B,
 * the multiplicity, the assembled Jacobi diagonal and the gather-scatter
 * groups, all inside `d_workspace` (device, 256-byte aligned, `bytes` >=
 * sem_mesh_workspace_bytes).  Waits for `stream` before returning (it checks
 * det J).  Returns SEM_ERR_MESH if det J <= 0 at any GLL point,
 * SEM_ERR_WORKSPACE if the workspace is too small or misaligned. */
int sem_mesh_create(const sem_mesh_desc *desc, void *d_workspace, size_t bytes,
                    void *stream, sem_mesh **out);
int sem_mesh_destroy(sem_mesh *mesh);
int sem_mesh_get_info(const sem_mesh *mesh, sem_mesh_info *info);

/* Physical coordinates of the GLL points: xyz[a][e][p] (device, 3*nloc). */
int sem_mesh_coords(const sem_mesh *mesh, double *xyz, void *stream);

/* Copies of mesh arrays (device destinations, nloc values each):
 * which = 0: mass B; 1: multiplicity; 2: inverse assembled Jacobi diagonal
 * (0 on Dirichlet nodes); 3..8: geometric factor rr, ss, tt, rs, rt, st
 * (E-layout, nloc values each). */
int sem_mesh_field(const sem_mesh *mesh, int which, double *dst, void *stream);

/* Local (unassembled) stiffness w = A_L u, element by element:
 *   u_r = D u, u_s, u_t along the three directions; v = G (u_r,u_s,u_t);
 *   w = D^T v_r + D^T v_s + D^T v_t.
 * u, w: device, nloc values of `dtype`:
 *  - SEM_F64: FP64 fields, FP64 arithmetic;
 *  - SEM_F32: FP32 fields, FP32 arithmetic (mesh built with SEM_GEOM_F32);
 *  - SEM_F64_PAIR: FP64 fields (double in, double out) but NOT FP64
 *    arithmetic: every value is carried as an unevaluated sum of two floats
 *    (double-float, 48 significant bits against FP64's 53) and the
 *    contractions run on the FP32 pipes with exact product and sum error
 *    terms (mesh built with SEM_GEOM_PAIR).  Error about 2^-42 of the
 *    line-wise magnitudes |D^T||G||D||u| (FP64: ~2^-50): within 1e-12 of
 *    the FP64 result in the relative 2-norm on fields without strong
 *    cancellation, up to ~1e-11 on smooth fields where A u cancels.  For
 *    residuals of iterative refinement, whose error only has to stay far
 *    below the solver tolerance.  Each element is scaled by a power of two
 *    (exact) before the split, so any magnitude is handled; values below
 *    2^-74 of the element's largest keep 24 bits, below 2^-126 of it they
 *    count as zero; FP64 denormals count as zero; an Inf or NaN in an
 *    element makes its whole output NaN.
 * u and w must not overlap. */
int sem_ax(const sem_mesh *mesh, const void *u, void *w, int dtype, void *stream);

/* Local Helmholtz operator w = h1 A_L u + h2 B u (FP64). */
int sem_helmholtz(const sem_mesh *mesh, double h1, double h2, const double *u, double *w,
                  void *stream);

/* Gather-scatter (direct stiffness summation) in place: every copy of a
 * shared global node receives the sum of all its copies, accumulated in
 * ascending local index; with apply_mask != 0 the nodes on Dirichlet faces
 * are then set to 0.  u: device, nloc values of `dtype`. */
int sem_dssum(const sem_mesh *mesh, void *u, int dtype, int apply_mask, void *stream);

/* Scatter a global-node vector to E-layout: u_loc[l] = u_glob[gid(l)],
 * gid = I + Gx (J + Gy K) of the box numbering (G_a = nel_a N, plus 1 on a
 * non-periodic axis).  Device pointers, FP64. */
int sem_scatter(const sem_mesh *mesh, const double *u_glob, double *u_loc, void *stream);

/* Unique-node inner product <a, b> = sum_l a_l b_l / mult_l of continuous
 * E-layout fields, FP64, written to *d_result (device).  Deterministic. */
int sem_glsc3(const sem_mesh *mesh, const double *a, const double *b, double *d_result,
              void *d_scratch, size_t scratch_bytes, void *stream);

/* sem_glsc3 without a scratch argument, for callers that cannot allocate
 * device memory: host codes whose device memory is owned by their own pool
 * or framework allocator (a library must not allocate behind it), fixed-
 * budget embedded or plugin contexts, and time-step loops that cannot take
 * the implicit device synchronisation or the failure point of cudaMalloc /
 * cudaFree.  The paper has no counterpart; this is a library convenience.
 *  - Scratch: a file-scope device array of 8448 bytes (1024 block partials
 *    and a counter), held by every device that loads the library until the
 *    process exits.  The reduction always runs 1024 blocks, so any mesh the
 *    library accepts fits (the same meshes as sem_glsc3); the call still
 *    checks the need against the array and rejects it with
 *    SEM_ERR_WORKSPACE.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and give wrong results; serialise
 *    them.  The counter is cleared on every call.
 *  - No cudaMalloc, cudaFree or allocating library routine is called.
 * Result and arguments as sem_glsc3. */
int sem_glsc3_noalloc(const sem_mesh *mesh, const double *a, const double *b, double *d_result,
                      void *stream);

/* Jacobi-preconditioned conjugate gradients on the assembled system
 * M Q Q^T (h1 A_L + h2 B) x = b (M: Dirichlet mask).  b must be continuous
 * and zero on Dirichlet nodes.  Stops when ||r|| <= tol ||b|| (tol_is_
 * relative) or ||r|| <= tol, with ||.|| the unique-node norm.
 * precision = SEM_PCG_F64: all FP64.
 * precision = SEM_PCG_MIXED: FP64 iterative refinement around FP32 PCG
 *   (FP32 operator and vectors, FP32 accumulation): every time the FP32
 *   residual has fallen by inner_tol, the FP32 increment is added to the FP64
 *   solution and the FP64 residual b - A x is recomputed; the outer dot
 *   products and the solution are FP64.  Requires SEM_GEOM_F32 in the mesh.
 * precision = SEM_PCG_F64_PAIR: FP64 vectors, dot products and updates
 *   with the operator evaluated in double-float arithmetic (as sem_ax
 *   SEM_F64_PAIR; error ~2^-42 of the line-wise magnitudes): not an FP64
 *   solve -- it converges in the FP64 solver's iterations and its solution
 *   meets the tolerance in the FP64 true residual, but differs from the FP64
 *   solution by the operator's error times the condition number.  Poisson
 *   only (h1 = 1, h2 = 0); requires SEM_GEOM_PAIR in the mesh. */
#define SEM_PCG_F64 0
#define SEM_PCG_MIXED 1
#define SEM_PCG_F64_PAIR 2
typedef struct {
    double tol;            /* stopping tolerance */
    int tol_is_relative;   /* 1: relative to ||b||, 0: absolute */
    int max_iter;          /* total inner iterations allowed */
    int precision;         /* SEM_PCG_F64 or SEM_PCG_MIXED */
    double inner_tol;      /* SEM_PCG_MIXED: inner relative tolerance (e.g. 1e-4) */
    double h1, h2;         /* operator h1 A + h2 B; Poisson: h1 = 1, h2 = 0 */
    int check_every;       /* iterations between host convergence checks (0 = 16) */
    int use_initial_guess; /* 1: x holds x0 on entry; 0: start from x = 0 */
    int profile;           /* 1: time the operator kernels with CUDA events
                              recorded on `stream` (fills ax_ms / gs_ms) */
    const double *dinv;    /* optional device array (nloc): inverse Jacobi diagonal to
                              use instead of the mesh's Poisson one (FP64 solves) */
    int mixed_restart;     /* SEM_PCG_MIXED: 0 (default) keeps the FP32 search
                              direction across FP64 refinements (the FP64 true
                              residual replaces the FP32 one, p is rescaled); 1
                              restarts the inner CG at every refinement */
    const struct sem_schwarz *schwarz;  /* SEM_PCG_MIXED, Poisson: the inner FP32 solve
                              is flexible CG preconditioned by this hybrid Schwarz
                              object (see sem_schwarz_create; built on the same
                              mesh, else SEM_ERR_INVALID_ARG), restarted at every
                              refinement; NULL: Jacobi */
    int coarse_iters;      /* Schwarz: coarse-level CG iterations per application
                              (0: one-level Schwarz; 3 suffice on the channel) */
    double coarse_tol;     /* Schwarz: coarse-level relative tolerance (0 = 1e-2) */
    int outer_pair;        /* SEM_PCG_MIXED: 1 forms the FP64 outer residual b - A x
                              with the operator in FP32-pair arithmetic (SEM_F64_PAIR,
                              mesh built with SEM_GEOM_PAIR, else
                              SEM_ERR_INVALID_ARG): ~2^-42 of the line-wise
                              magnitudes instead of FP64 rounding, 5x faster on
                              GB300; 0 (default): the FP64 operator */
    const struct sem_schwarz *schwarz_mid;  /* with schwarz: the intermediate level of the
                              Schwarz multigrid (a Schwarz object built on the
                              order-M mesh of the same elements, M < N, see
                              sem_schwarz_apply3); NULL: two levels */
    double mid_weight;     /* its weight w_M (0 = 0.15) */
    double inner_adapt;    /* SEM_PCG_MIXED: theta > 0 lets a refinement round stop
                              once the outer target is within reach: its inner
                              relative tolerance is max(inner_tol, min(0.5,
                              theta * target / ||r||)), with target the outer
                              stopping norm and r the FP64 residual the round
                              starts from (a guess already near the target needs
                              a short round, not a reduction by inner_tol);
                              0 (default): inner_tol every round.  The FP64 true
                              residual still decides convergence. */
    int krylov;            /* SEM_PCG_MIXED: inner Krylov method, SEM_KRYLOV_CG (default:
                              Jacobi-PCG, or flexible CG with a Schwarz preconditioner)
                              or SEM_KRYLOV_FGMRES: flexible restarted GMRES (the
                              paper's pressure solver, Sec. 3.1), one cycle of at most
                              gmres_restart iterations per refinement round (the
                              restart is the refinement: the next cycle starts from the
                              FP64 true residual), preconditioned by the Schwarz
                              object(s) or the Jacobi diagonal; Arnoldi in FP32 with
                              classical Gram-Schmidt and a second pass where the first
                              cancelled all but 1 % of the vector */
    int gmres_restart;     /* SEM_KRYLOV_FGMRES: cycle length, 1..128 (0 = 30); the
                              scratch grows by 2 gmres_restart + 2 FP32 vectors */
} sem_pcg_opts;
#define SEM_KRYLOV_CG 0
#define SEM_KRYLOV_FGMRES 1

typedef struct {
    int iters;             /* total (inner) CG iterations */
    int outer_iters;       /* refinement steps (SEM_PCG_MIXED), else 0 */
    int status;            /* same as the return value */
    double rel_res;        /* final ||r|| / ||b|| (FP64 true residual for MIXED) */
    double abs_res;        /* final ||r|| */
    double bnorm;          /* ||b|| */
    double wall_ms;        /* host wall time of the call */
    double ax_ms;          /* profile: summed device time of operator kernels */
    double gs_ms;          /* profile: summed device time of gather-scatter kernels */
    int ax_launches;       /* operator kernel launches (MIXED: inner FP32 ones) */
    int kernel_launches;   /* all kernel launches of the call */
    double outer_ax_ms;    /* MIXED + profile: device time of the FP64 outer operators */
    int outer_ax_launches; /* MIXED: FP64 outer operator launches */
    double init_rel_res;   /* ||b - A x0|| / ||b|| of the initial guess */
} sem_pcg_stats;

/* Scratch bytes sem_pcg_solve needs (device). */
size_t sem_pcg_scratch_bytes(const sem_mesh *mesh, const sem_pcg_opts *opts);

/* Solve; b, x device FP64 E-layout (x: initial guess if use_initial_guess,
 * solution on return, continuous).  Waits for `stream` (it reads the
 * convergence flag every check_every iterations) and fills *stats (host).
 * Returns SEM_OK, SEM_ERR_NOT_CONVERGED (x and stats still valid),
 * SEM_ERR_NAN, SEM_ERR_WORKSPACE, SEM_ERR_TIMEOUT or SEM_ERR_CUDA. */
int sem_pcg_solve(const sem_mesh *mesh, const double *b, double *x, const sem_pcg_opts *opts,
                  sem_pcg_stats *stats, void *d_scratch, size_t scratch_bytes, void *stream);

/* The same solve with HOST buffers: copies b (host, nloc doubles; pinned
 * memory makes the copy asynchronous) to the device, solves, and copies the
 * solution back to x (host; its contents on entry are the initial guess when
 * use_initial_guess).  d_scratch must hold sem_pcg_host_scratch_bytes. */
size_t sem_pcg_host_scratch_bytes(const sem_mesh *mesh, const sem_pcg_opts *opts);
int sem_pcg_solve_host(const sem_mesh *mesh, const double *h_b, double *h_x, const sem_pcg_opts *opts,
                       sem_pcg_stats *stats, void *d_scratch, size_t scratch_bytes, void *stream);

/* ---- Navier-Stokes building blocks (section 3, Eq. 1) --------------------
 * All need a mesh built with SEM_GEOM_RX; device FP64 E-layout arrays. */

/* Collocation gradient g[m][l] = sum_a (dr_a/dx_m) (D_a f)[l], m = x, y, z
 * (g: 3*nloc).  Element-local (not assembled). */
int sem_gradient(const sem_mesh *mesh, const double *f, double *g, void *stream);

/* Advection term nl[c] = -sum_m u[m] d u[c]/dx_m (u, nl: 3*nloc),
 * collocation, no dealiasing. */
int sem_advect(const sem_mesh *mesh, const double *u, double *nl, void *stream);

/* Local weak divergence w_i = int grad(phi_i) . F (F: 3*nloc) by GLL
 * quadrature: sum_a D_a^T [B sum_m (dr_a/dx_m) F_m].  Not assembled. */
int sem_weak_div(const sem_mesh *mesh, const double *F, double *w, void *stream);

/* Incompressible Navier-Stokes time stepper on a fully periodic box mesh
 * (section 3.1: velocity-pressure splitting, Krylov pressure solve each step,
 * CG for the velocity).  Scheme: BDF_k / EXT_k, k = min(step+1, 2), P_N-P_N:
 *   F = sum_j (b_j/dt) u^{n+1-j} + sum_j a_j NL^{n+1-j},  NL = -(u.grad)u
 *   A p = Q Q^T wdiv(F) - mean        (singular; p shifted to zero mean)
 *   (nu A + (b0/dt) B) u_c = Q Q^T [B (F_c - dp/dx_c)],  nu = 1/Re
 * The state lives in a caller workspace; pressures of the last three steps
 * are kept (for extrapolated or learned initial guesses). */
typedef struct sem_ns sem_ns;
size_t sem_ns_workspace_bytes(const sem_mesh *mesh);
int sem_ns_create(const sem_mesh *mesh, double Re, void *d_workspace, size_t bytes, void *stream,
                  sem_ns **out);
int sem_ns_destroy(sem_ns *ns);
/* Set the velocity (device, 3*nloc, continuous), clear the history. */
int sem_ns_set_velocity(sem_ns *ns, const double *u, void *stream);
/* Copy a state field to dst (device, nloc): 0..2 velocity u^n, 3 pressure
 * p^n, 4 pressure p^{n-1}, 5 pressure p^{n-2}, 6 the last pressure right-
 * hand side (assembled, zero mean), 7..9 velocity u^{n-1}, 10..12 advection
 * term NL^{n-1}, 13..15 velocity u^{n-2}, 16..18 NL^{n-2}.  sem_ns_set writes
 * the same slots (checkpoint restore); with sem_ns_get_steps /
 * sem_ns_set_steps they hold the whole state. */
int sem_ns_get(const sem_ns *ns, int which, double *dst, void *stream);
int sem_ns_set(sem_ns *ns, int which, const double *src, void *stream);
int sem_ns_get_steps(const sem_ns *ns);
int sem_ns_set_steps(sem_ns *ns, int steps);
/* Time scheme and advection form (defaults: order 2, collocation).
 * order 1..3: step n uses BDF_k / EXT_k with k = min(n+1, order); order 3 is
 * the BDF3 / EXT3 pair of the high-order splitting the paper cites for Neko
 * (section 3.1): b0 = 11/6, b = (3, -3/2, 1/3), a = (3, -3, 1).
 * dealias != 0: the advection term is integrated exactly on M = 3(N+1)/2
 * Gauss-Legendre points per direction (the 3/2 rule) in its weak form
 * int phi_i (u.grad)u_c, then assembled and divided by the assembled mass;
 * d_dealias (device, 256-byte aligned, >= sem_ns_dealias_bytes) receives the
 * fine-point metric factors (9 doubles per Gauss point) and must stay alive
 * while the state is used.  N <= 9.  Stream-ordered. */
size_t sem_ns_dealias_bytes(const sem_mesh *mesh);
int sem_ns_set_scheme(sem_ns *ns, int order, int dealias, void *d_dealias, size_t bytes, void *stream);
/* The state's advection term of u (device, 3*nloc, continuous) into nl
 * (device, 3*nloc): -(u.grad)u by collocation, or its dealiased form. */
int sem_ns_advect(const sem_ns *ns, const double *u, double *nl, void *stream);
/* Scratch for sem_ns_step with these solver options. */
size_t sem_ns_scratch_bytes(const sem_ns *ns, const sem_pcg_opts *popts, const sem_pcg_opts *vopts);
/* One time step.  popts / vopts: pressure / velocity solver options (the
 * velocity solves use h1 = nu, h2 = b0/dt and their own Jacobi diagonal;
 * those fields of vopts are ignored).  Initial guess of the pressure:
 * p_guess (device, nloc) if non-NULL, else the previous pressure when
 * popts->use_initial_guess, else zero.  pstats: 1 entry, vstats: 3 entries
 * (host).  Waits for `stream`. */
int sem_ns_step(sem_ns *ns, double dt, const sem_pcg_opts *popts, const sem_pcg_opts *vopts,
                const double *p_guess, sem_pcg_stats *pstats, sem_pcg_stats *vstats, void *d_scratch,
                size_t scratch_bytes, void *stream);
/* The same step in two calls, so that an initial guess can be built from
 * the new pressure right-hand side (slot 6) before the solves:
 * sem_ns_step_begin forms the advection term, the forcing and the pressure
 * right-hand side; sem_ns_step_finish does the solves and the history
 * update (arguments as sem_ns_step). */
int sem_ns_step_begin(sem_ns *ns, double dt, void *stream);
int sem_ns_step_finish(sem_ns *ns, const sem_pcg_opts *popts, const sem_pcg_opts *vopts,
                       const double *p_guess, sem_pcg_stats *pstats, sem_pcg_stats *vstats,
                       void *d_scratch, size_t scratch_bytes, void *stream);
/* Kinetic energy (1/2V) int |u|^2 and its GLL quadrature, on the host
 * (waits for `stream`). */
int sem_ns_kinetic_energy(const sem_ns *ns, double *energy, void *d_scratch, size_t scratch_bytes,
                          void *stream);

/* ---- BF16 GEMM on the tensor cores (element-local network) ---------------
 * C[M x N] = act(A . B^T + bias): A [M x K] and B [N x K] row-major BF16
 * (device, 16-byte aligned, K contiguous), FP32 accumulation; act 0 =
 * identity, 1 = ReLU; bias [N] FP32 or NULL; C32 (FP32) and/or C16 (BF16)
 * row-major with leading dimension ldc (>= N, multiple of 4).  M % 128 == 0,
 * N % 128 == 0, K % 64 == 0.  d_err: device int that receives a non-zero code
 * if a bounded wait gave up (check it with a stream synchronisation).
 * Stream-ordered, asynchronous.  Not from the paper: the learned initial
 * guess of the pressure solve uses it. */
int sem_gemm_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int act, float *C32,
                  void *C16, int ldc, int *d_err, void *stream);
/* The same product with split-K for small outputs: when the 128 x BN output
 * tiles alone fill fewer CTAs than the GPU has SMs, K is cut into up to 16
 * slices (at least 8 K-blocks of 64 each), each slice's FP32 tile is written
 * to d_work, and a second kernel sums the slices in slice order
 * (deterministic), adds the bias and applies the activation.  d_work:
 * device, 16-byte aligned, work_bytes >= sem_gemm_bf16_splitk_work_bytes
 * for the full 16 slices (fewer fit a smaller work space); NULL: no split.
 * Used for the network's weight gradients (M x N <= 256 x 2048, K = the
 * rows). */
size_t sem_gemm_bf16_splitk_work_bytes(int M, int N, int K);
int sem_gemm_bf16_splitk(const void *A, const void *B, int M, int N, int K, const float *bias, int act,
                         float *C32, void *C16, int ldc, void *d_work, size_t work_bytes, int *d_err,
                         void *stream);

/* ---- Element-local network for the learned initial guess ----------------
 * Not from the paper.  Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per row
 * (one row per element); loss (1/(2 R O)) sum (Y - T)^2 over the first R
 * rows and O outputs; Adam.  Training and inference GEMMs run on
 * sem_gemm_bf16 (BF16 operands, FP32 accumulation); master parameters,
 * gradients and Adam moments are FP32 in one flat array ordered W1 [H x I],
 * b1 [H], W2 [H x H], b2 [H], W3 [O x H], b3 [O].  I, H, O and the row
 * counts passed below must be multiples of 128 (pad with zeros). */
typedef struct sem_mlp sem_mlp;
size_t sem_mlp_workspace_bytes(int n_in, int n_hidden, int n_out, int max_rows);
int sem_mlp_create(int n_in, int n_hidden, int n_out, int max_rows, void *d_workspace, size_t bytes,
                   sem_mlp **out);
int sem_mlp_destroy(sem_mlp *mlp);
size_t sem_mlp_num_params(const sem_mlp *mlp);
/* Parameters from / to a host FP32 array of sem_mlp_num_params values;
 * set also clears the Adam moments. */
int sem_mlp_set_params(sem_mlp *mlp, const float *host, void *stream);
int sem_mlp_get_params(const sem_mlp *mlp, float *host, void *stream);
int sem_mlp_get_grads(const sem_mlp *mlp, float *host, void *stream);
/* Y [rows x O] (device FP32) from X [rows x I] (device BF16). */
int sem_mlp_forward(sem_mlp *mlp, const void *X, int rows, float *Y, void *stream);
/* Forward and backward on X, T [rows x O] (device FP32); gradients kept in
 * the network; *loss (host) over rows_real rows and outs_real outputs.
 * Waits for `stream`. */
int sem_mlp_grad(sem_mlp *mlp, const void *X, const float *T, int rows, int rows_real, int outs_real,
                 double *loss, void *stream);
/* Forward and backward with the energy-norm loss of a guess network on
 * `mesh` (one row per element, output q = the element's point q):
 *   L = (1 / (2 E npt)) sum_e d_e^T (A_e + lambda B_e) d_e
 * over the E elements and npt points, with d = Y - T (assembled = 0) or,
 * assembled = 1, d = M^-1 Q Q^T (Y - T): the error of the averaged,
 * continuous correction the guess uses (sem_guess_apply), so that the
 * disagreement of neighbouring elements is part of the loss (gradient
 * Q Q^T M^-1 (A_L + lambda B) d).  A_e: element stiffness matrix, the local
 * operator of sem_ax, here in FP32 on the mesh's FP32 geometric factors;
 * B_e: diagonal mass; the sums of copies in FP32.  Errors of high spatial
 * frequency, which the solver sees amplified in its residual, weigh more
 * than in the plain mean square; lambda B keeps the element-wise constants
 * (the null space of A_e) in the loss.  X [rows x I] BF16, T [rows x O] FP32
 * (row e = element e, rows >= E, O >= npt); work: device, >= 2 nloc floats
 * (caller-owned).  Requires SEM_GEOM_F32 in the mesh; lambda >= 0.  Waits
 * for `stream`. */
int sem_mlp_grad_energy(sem_mlp *mlp, const sem_mesh *mesh, const void *X, const float *T, int rows,
                        double lambda, int assembled, float *work, size_t work_floats, double *loss,
                        void *stream);
/* One Adam step with the stored gradients. */
int sem_mlp_adam(sem_mlp *mlp, double lr, double beta1, double beta2, double eps, void *stream);

/* The guess corrects the cubic extrapolation p_ext = 3 p1 - 3 p2 + p3 of the
 * last three pressures.  sem_guess_residual: r = b - M Q Q^T A_L p_ext
 * (FP64; work: nloc doubles, receives p_ext).  The error the guess must
 * remove, e = p - p_ext, satisfies A e = r. */
int sem_guess_residual(const sem_mesh *mesh, const double *b, const double *p1, const double *p2,
                       const double *p3, double *r, double *work, void *stream);
/* The same residual with the operator in FP32-pair arithmetic (as sem_ax
 * SEM_F64_PAIR: error ~2^-42 of the line-wise magnitudes, plenty for a
 * feature that is rounded to BF16); requires SEM_GEOM_PAIR in the mesh. */
int sem_guess_residual_pair(const sem_mesh *mesh, const double *b, const double *p1, const double *p2,
                            const double *p3, double *r, double *work, void *stream);
/* Features for every element e (row e of X, BF16, ldx >= 4 npt):
 * (p1 - p2)/sd, (p2 - p3)/sd, r/sr and, with p4 (the pressure four steps
 * back) given, the previous step's extrapolation error (third difference)
 * (p1 - 3 p2 + 3 p3 - p4)/s4, else p1/s4, at the element's points. */
int sem_guess_features(const sem_mesh *mesh, const double *p1, const double *p2, const double *p3,
                       const double *p4, const double *r, double sd, double sr, double s4, void *X, int ldx,
                       void *stream);
/* Training target T[e][q] = (p - p_ext) / se (FP32, ldt >= npt). */
int sem_guess_target(const sem_mesh *mesh, const double *p, const double *p1, const double *p2,
                     const double *p3, double se, float *T, int ldt, void *stream);
/* Guess = (Q Q^T g) / mult with g = p_ext + se Y (continuous FP64 E-layout). */
int sem_guess_apply(const sem_mesh *mesh, const float *Y, int ldy, const double *p1, const double *p2,
                    const double *p3, double se, double *guess, void *stream);

/* ---- Batched solves ------------------------------------------------------
 * nsolve independent systems (meshes[i], b[i], x[i]; device FP64 E-layout;
 * meshes may differ in size and order) solved together by the mixed solver
 * (opts->precision must be SEM_PCG_MIXED with the Jacobi inner solver, every
 * mesh built with SEM_GEOM_F32, x starts from 0).  One CUDA graph, launched
 * once: every solve is a parallel branch whose rounds (check_every FP32
 * iterations plus one FP64 refinement stage) repeat in a device-side WHILE
 * loop until the solve has converged, failed, spent its round budget
 * (max_iter / check_every + 64) or met a device timeout; all decisions are
 * taken on the device, so each solve advances at its own pace and the host
 * waits once.  The branches carry scheduling priorities by estimated work
 * (local points x elements along an axis x N; the smallest the greatest
 * priority, spread over the device's priority levels): small solves are
 * served first.  stats[i] (host) as for sem_pcg_solve, with wall_ms = device
 * time from the start of the graph to the end of solve i's last round,
 * ax_launches = the rounds it ran.  Waits for `stream`.  Returns SEM_OK when
 * all converged; SEM_ERR_UNSUPPORTED for other precisions, a Schwarz
 * preconditioner, outer_pair or an initial guess. */
size_t sem_pcg_batched_scratch_bytes(const sem_mesh *const *meshes, int nsolve, const sem_pcg_opts *opts);
int sem_pcg_solve_batched(const sem_mesh *const *meshes, int nsolve, const double *const *b,
                          double *const *x, const sem_pcg_opts *opts, sem_pcg_stats *stats,
                          void *d_scratch, size_t scratch_bytes, void *stream);
/* The same batched solve with the hybrid Schwarz preconditioner (section
 * 3.1's pressure preconditioner) per solve: schwarz[i] built on meshes[i]
 * (sem_schwarz_create), coarse_iters / coarse_tol from opts (opts->schwarz
 * stays NULL).  The inner FP32 solve of each refinement is flexible CG,
 * restarted from the new FP64 residual at every refinement; the coarse CG
 * runs as separate launches (no grid barrier: the solves' graph branches run
 * concurrently).  Scratch as sem_pcg_batched_scratch_bytes.
 * SEM_ERR_INVALID_ARG if schwarz[i] was built on another mesh. */
int sem_pcg_solve_batched_schwarz(const sem_mesh *const *meshes, const struct sem_schwarz *const *schwarz,
                                  int nsolve, const double *const *b, double *const *x, const sem_pcg_opts *opts,
                                  sem_pcg_stats *stats, void *d_scratch, size_t scratch_bytes, void *stream);

/* ---- Autotuner of the operator launch shape -------------------------------
 * Times the operator of `mesh` (precision dtype, plain or fused CG form) and
 * keeps the fastest launch shape for the mesh's order N in the library's
 * launch table (process-wide, all meshes of that order use it).  FP32:
 * pipeline depths {1, 2, 3} x resident-CTAs-per-SM caps {none, 1, 2, 4} x
 * elements per CTA {1, 2, 4} (the block shape; groups of elements where
 * (N+1)^2 threads leave warps partly empty: 2 <= N <= 9, (N+1)^2 not a
 * multiple of 32, general or BF16 factors); FP64: the CTA cap only.
 * Scratch: device, sem_autotune_scratch_bytes.  Waits for `stream`.  Not
 * from the paper. */
#define SEM_TUNE_MAX_CONFIGS 48
typedef struct {
    int best_stages, best_cap, best_epc;
    float best_ms;
    int configs;
    int stages[SEM_TUNE_MAX_CONFIGS], caps[SEM_TUNE_MAX_CONFIGS], epcs[SEM_TUNE_MAX_CONFIGS];
    float ms[SEM_TUNE_MAX_CONFIGS];
} sem_tune_result;
size_t sem_autotune_scratch_bytes(const sem_mesh *mesh);
int sem_autotune_operator(const sem_mesh *mesh, int dtype, int fused_cg, void *d_scratch, size_t bytes,
                          void *stream, sem_tune_result *out);
/* Set the launch shape of `mesh`'s order for dtype / fused_cg (as the
 * autotuner would, without timing): stages 1..3, per_sm_cap >= 0 (0 = the
 * occupancy limit), epc 1, 2 or 4 (elements per CTA; used by the FP32
 * operator where it builds groups, else 1).  SEM_ERR_INVALID_ARG outside. */
int sem_autotune_set(const sem_mesh *mesh, int dtype, int fused_cg, int stages, int per_sm_cap, int epc);
/* Back to the default launch shapes (2 stages, occupancy-limited, 1 element
 * per CTA). */
int sem_autotune_reset(void);

/* ---- Hybrid Schwarz preconditioner of the pressure solve ------------------
 * Section 3.1: the pressure is solved with a Krylov method and a hybrid-
 * Schwarz multigrid preconditioner (the SEM overlapping Schwarz / fast-
 * diagonalisation method).  Two additive levels, symmetric, FP32:
 *   z = sum_e R_e^T A_e^{-1} R_e r  +  P A_c^{-1} P^T r
 * R_e: element e extended by one GLL point into each neighbour; A_e the
 * separable operator of that subdomain (1-D stiffness and mass along each
 * direction from the mean edge lengths of the element and its neighbours,
 * homogeneous Dirichlet just beyond the overlap), inverted by fast
 * diagonalisation (exact for axis-aligned tensor-product meshes); P the
 * trilinear interpolation from the element vertices, A_c the N = 1 operator
 * (assembled at set-up into a 27-point stencil on the global vertices),
 * solved by up to coarse_iters Jacobi-CG iterations from 0, stopping early
 * when <r, D^-1 r> falls by coarse_tol^2 (0 iterations: no coarse level).
 * mesh: 2 <= N <= 9, built with SEM_GEOM_F32; coarse: the N = 1 mesh of the
 * same vertices and topology (its FP64 geometric factors give A_c).  Set-up
 * solves the 1-D eigenproblems on the host (cached by length and boundary
 * type), assembles A_c on the device and waits for `stream`.  The object
 * keeps pointers to both meshes; the workspace (sem_schwarz_workspace_bytes)
 * holds the tables, the extended local solutions (4 (N+3)^3 B per element)
 * and the coarse vectors.  Errors: SEM_ERR_INVALID_ARG (NULL, wrong coarse
 * mesh, mesh without FP32 factors), SEM_ERR_UNSUPPORTED (N outside 2..9),
 * SEM_ERR_WORKSPACE. */
typedef struct sem_schwarz sem_schwarz;
size_t sem_schwarz_workspace_bytes(const sem_mesh *mesh, const sem_mesh *coarse);
int sem_schwarz_create(const sem_mesh *mesh, const sem_mesh *coarse, void *d_workspace, size_t bytes,
                       void *stream, sem_schwarz **out);
int sem_schwarz_destroy(sem_schwarz *sw);
/* Number of distinct 1-D eigenproblems solved at set-up. */
int sem_schwarz_problems(const sem_schwarz *sw);
/* The set-up's 1-D problem of one direction of an extended element (host
 * computation, no GPU; the fast-diagonalisation factors of the local solves
 * of the section 3.1 preconditioner): stiffness and mass of the left neighbour, the
 * element and the right neighbour (lengths hL, h, hR > 0) on the N + 3
 * extended GLL points; flags bit 0: a left neighbour exists, bit 1: a right
 * one, bit 2: the element's low face is Dirichlet, bit 3: its high face (such
 * points are decoupled as identity rows).  Writes S[(N+3)^2] (row-major, row
 * = point, column = mode; S^T B S = I) and lambda[N+3] (A S = B S Lambda,
 * unsorted).  SEM_ERR_UNSUPPORTED outside 2 <= N <= 9, SEM_ERR_INVALID_ARG
 * for NULL outputs, lengths <= 0 or unknown flags. */
int sem_schwarz_fdm_1d(int N, double h, double hL, double hR, int flags, double *S, double *lambda);
/* The coarse operator the set-up assembles (the preconditioner's trilinear
 * coarse level, section 3.1), computed on the host by the same code (no
 * GPU): from the N = 1 geometric factors G[E][6][8] (FP64,
 * rr, ss, tt, rs, rt, st at the element vertices, quadrature weights
 * included; E = nel[0] nel[1] nel[2], elements x fastest), the 27-point
 * stencil sten[27][nv] (offset (ox, oy, oz) in {-1,0,1}^3 at index
 * (ox+1) + 3(oy+1) + 9(oz+1); vertex v = vx + nv0 (vy + nv1 vz), nv_a =
 * nel_a + (periodic_a ? 0 : 1), nv = nv0 nv1 nv2) with rows and columns of
 * Dirichlet vertices (faces bits as in sem_mesh_desc) zeroed, and cdinv[nv]
 * = 1 / assembled diagonal (0 on Dirichlet vertices).  FP32 outputs, host
 * arrays owned by the caller.  SEM_ERR_INVALID_ARG for NULL or nel < 1. */
int sem_schwarz_coarse_operator(const int *nel, const int *periodic, int faces, const double *G, float *sten,
                                float *cdinv);
/* The local-solve kernel's line tables for order N (host, no GPU; a GB300
 * scheduling detail, not from the paper): for each
 * of the three line directions (along I, J, K), *slots = 32 LPT entries (LPT
 * lines per lane) holding the line dealt to (group q = slot / 32, lane =
 * slot % 32), or -1; line id c1 + (N+3) c2 with (c1, c2) = (J, K), (I, K),
 * (I, J).  The I and J tables spread the lines' shared-memory banks; the K
 * passes use the natural order (slot = line).  *pj, *pk: the shared-block
 * strides the tables were built for.  out needs 3 *slots shorts (cap: its
 * length; SEM_ERR_WORKSPACE if smaller). */
int sem_schwarz_line_table(int N, short *out, int cap, int *slots, int *pj, int *pk);
/* z = M r (device FP32 E-layout, r continuous and zero on Dirichlet nodes;
 * z continuous, every copy of a node bit-identical, zero on Dirichlet
 * nodes).  Stream-ordered, no host synchronisation; three kernels (local
 * solves, the cooperative coarse CG when coarse_iters > 0, overlap sums).
 * The coarse CG's grid barriers wait at most 1 s; a timeout is recorded in
 * the mesh's error word (reported as SEM_ERR_TIMEOUT by the solver). */
int sem_schwarz_apply(const sem_schwarz *sw, const float *r, float *z, int coarse_iters, double coarse_tol,
                      void *stream);

/* The three-level Schwarz multigrid (section 3.1 names a hybrid-Schwarz
 * multigrid; its depth is read here as the paper's solver, Neko, uses it:
 * fine order N, an intermediate order M, the trilinear coarse level):
 *   z = S_N r + w_M P_M S_M P_M^T r + P A_c^{-1} P^T r,
 * S_N r + P A_c^{-1} P^T r as sem_schwarz_apply(sw, ...); S_M the
 * overlapping Schwarz of `mid` (a Schwarz object built on the order-M mesh
 * of the same elements and topology, M < N; its coarse level is not used);
 * P_M element-wise interpolation from the order-M GLL points to the order-N
 * ones (exact for degree <= M), P_M^T r = Q_M Q_M^T J^T (r / mult) masked.
 * The levels are added (symmetric); w_M > 0 damps the intermediate level,
 * whose correction overlaps the fine one (0.15 on the channel).  r, z:
 * device FP32 E-layout as sem_schwarz_apply; d_work: device, 256-byte
 * aligned, sem_schwarz_mid_work_bytes(mid) bytes.  Stream-ordered.
 * SEM_ERR_INVALID_ARG for a mismatched `mid` or w_M <= 0, SEM_ERR_WORKSPACE
 * for missing work space. */
size_t sem_schwarz_mid_work_bytes(const sem_schwarz *mid);
int sem_schwarz_apply3(const sem_schwarz *sw, const sem_schwarz *mid, double mid_weight, const float *r, float *z,
                       int coarse_iters, double coarse_tol, void *d_work, size_t bytes, void *stream);

/* ---- Performance model for splitting one problem over devices -----------
 * Section 4.1 (Eq. 2-7): a homogeneous cost C (here: element-iterations of a
 * solve) split over ndev devices; device i computes C_i at its best
 * performance P_opt[i] (cost per second) and holds at most C_max[i] (C_max
 * NULL or an entry <= 0: unlimited).  T_min = min over splits with
 * sum C_i = C, C_i <= C_max[i] of max_i C_i / P_opt[i]: C / sum P_opt when
 * the proportional split fits every capacity, else the devices whose
 * capacity binds are filled and the others share the rest in proportion to
 * P_opt (exact minimiser).  Writes *T_min and C_split[ndev] (host).  Returns
 * SEM_ERR_INVALID_ARG (ndev < 1, a P_opt <= 0, C < 0) or SEM_ERR_WORKSPACE
 * (the capacities hold less than C).  Host computation, no GPU. */
int sem_perf_model(int ndev, const double *P_opt, const double *C_max, double C, double *T_min,
                   double *C_split);

/* Read and clear the mesh's device error word after waiting for `stream`:
 * *code = 0 if no kernel on this mesh reported a bounded-wait timeout, 1 if
 * a bulk-copy (mbarrier) wait gave up, 2 if a grid-barrier wait gave up.
 * Every device wait of the library is bounded (1 s of global time); a
 * kernel that gives up records its code here (first writer wins), leaves
 * its loop and drains its own copies, so the context stays usable.  The
 * solvers (sem_pcg_solve*, sem_pcg_solve_batched, the sem_ns_* steps) clear
 * the word at entry and report a give-up of their own kernels as
 * SEM_ERR_TIMEOUT; other calls (sem_ax, sem_schwarz_apply, ...) leave it set
 * until it is read here.  While it is set, the grid barriers of the coarse
 * Schwarz level leave at once (sem_schwarz_apply then skips the coarse
 * correction). */
int sem_mesh_check_device_error(const sem_mesh *mesh, int *code, void *stream);

/* Self-test of the failure detection (not from the paper): launches a kernel
 * that waits, bounded by limit_s (0 < limit_s <= 10 s), on something nothing
 * will complete -- kind 0: an mbarrier whose transaction bytes no copy will
 * bring (the wait of every bulk-copy pipeline of the library); kind 1: two
 * CTAs on a grid barrier whose target exceeds the grid (the wait of the
 * cooperative coarse solve).  The wait gives up, writes its code (1 or 2)
 * into the mesh's error word and the kernel returns; no fault, no trap.
 * d_scratch: 16 bytes of 16-byte aligned device memory (kind 1; may be NULL
 * for kind 0).  Stream-ordered; read the result with
 * sem_mesh_check_device_error.  SEM_ERR_INVALID_ARG for an unknown kind or a
 * limit outside the range, SEM_ERR_WORKSPACE for missing scratch. */
int sem_wait_selftest(const sem_mesh *mesh, int kind, double limit_s, void *d_scratch, size_t bytes,
                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SEM_GB300_H */
