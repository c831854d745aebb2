/*
 * cgs.h -- C ABI of the B300 coarse-grid Schwarz solver.
 *
 * The library solves the N=1 element-vertex Poisson system A u = b of a pMG
 * pressure preconditioner with flexible PCG preconditioned by the two-level
 * overlapping Schwarz method of "Coarse Solvers for Exascale Solution of
 * Poisson Problems" (Ratnayaka, Fischer, Olson):
 *
 *   local part   l = sum_p R~_p^T A_p^{-1} R_p r            (Sec. 3, Eq. (4))
 *   box part     B_C s = J~ A_r^{-1} J~^T s,  J~ = W Q^T J_L  (Sec. 4)
 *   hybrid       z = l + B_C (r - A l)                      (Eq. (5))
 *   additive     z = sum_p R_p^T A_p^{-1} R_p r + B_C r     (Eq. (3))
 *
 * Conventions shared by every call
 *   - Meshes are trilinear hexahedra.  conn[8*e + k] is the vertex of local
 *     corner k = a + 2b + 4c, (a,b,c) in {0,1}^3 of the reference cube
 *     (lexicographic; Sec. 1).  xyz[3*v + d] is coordinate d of vertex v.
 *   - Vectors are float64 arrays of length nv in the caller's vertex order.
 *     Entries at Dirichlet vertices are ignored on input and written 0 on
 *     output.
 *   - "device" pointers are CUDA device (or managed) memory on the mesh's
 *     device; "host" pointers are ordinary CPU memory.  The library never
 *     keeps a caller pointer beyond the call.
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Calls are stream-ordered: they enqueue work and return without
 *     waiting unless the description says otherwise.  A mesh owns its scratch
 *     vectors, so two calls on the same mesh must not overlap on the GPU.
 *   - Every call returns a cgs_status; nothing is thrown across the ABI.
 *     cgs_last_error() returns a message for the calling thread's last error.
 */
#ifndef CGS_H
#define CGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cgs_ctx cgs_ctx;
typedef struct cgs_mesh cgs_mesh;

typedef enum {
    CGS_OK = 0,
    CGS_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad parameter   */
    CGS_ERR_INVALID_MESH = 2,  /* index out of range, Jacobian <= 0            */
    CGS_ERR_NOT_SPD = 3,       /* a local A_p or the reduced A_r not SPD       */
    CGS_ERR_NO_CONVERGENCE = 4,/* maxit reached before the tolerance           */
    CGS_ERR_BREAKDOWN = 5,     /* p.q <= 0, r.z <= 0 or a NaN in the iteration */
    CGS_ERR_OOM = 6,           /* device allocation failed                     */
    CGS_ERR_ADMISSION = 7,     /* setup would exceed the context's HBM budget  */
    CGS_ERR_TIMEOUT = 8,       /* a bounded device-side wait expired           */
    CGS_ERR_CUDA = 9           /* any other CUDA runtime error                 */
} cgs_status;

typedef enum {
    CGS_FP64 = 0,        /* every step in float64 (the plain form)                   */
    CGS_FP32_BULK = 1,   /* local solves, inner A apply, J~ and J~^T in float32;
                            reduced solve, outer A p, residual and dots in float64   */
    CGS_FP16_LOCAL = 2   /* as CGS_FP32_BULK, local inverses stored in float16 with
                            one float32 scale per subdomain                          */
} cgs_precision;

typedef enum {
    CGS_HYBRID = 0,      /* ASM_1 then ASM_2 (Eqs. (4), (5)), W_ov-weighted local sum */
    CGS_ADDITIVE = 1,    /* Eq. (3) with R~_p = R_p (symmetric)                         */
    CGS_RAS = 2          /* Eq. (3) with the restricted prolongation R~_p (Sec. 3, RAS):
                            a local solution keeps only the nodes of the original,
                            not grown, Omega_p, averaged where several original
                            subdomains store a node; not symmetric, so solve it
                            with a flexible method (the PCG here is flexible)     */
} cgs_form;

/* Reduced solver u_r = A_r^{-1} r_r (Sec. 2, the XX^T paragraph; Sec. 4). */
typedef enum {
    CGS_COARSE_AUTO = 0,   /* XX^T when n_r > CGS_COARSE_AUTO_XXT_NR, else dense     */
    CGS_COARSE_DENSE = 1,  /* explicit A_r^{-1}, one GEMV (n_r^2 entries)             */
    CGS_COARSE_XXT = 2     /* A_r^{-1} = X X^T with X sparse and A_r-conjugate under a
                              nested-dissection order of the box lattice: two sparse
                              passes t = X^T r_r, u_r = X t; needs n_r <= 65535      */
} cgs_coarse_solver;
#define CGS_COARSE_AUTO_XXT_NR 1500

/* The reduced operator A_r and its interpolation (Sec. 4). */
typedef enum {
    CGS_COARSE_OP_CELLWISE = 0, /* cell-wise assembly of Eq. (12) (3^3 stencil) with the
                                   averaged interpolant W Q^T J_L (default)            */
    CGS_COARSE_OP_GALERKIN = 1, /* the same interpolant, A_r = J~^T A J~ (5^3 stencil) */
    CGS_COARSE_OP_VERTEX = 2    /* vertex-based J: each node interpolated in the box
                                   cell holding it, A_r = J^T A J (5^3 stencil)         */
} cgs_coarse_operator;

typedef struct {
    int box[3];            /* b_x, b_y, b_z in [1, 1023]: box cells per axis over the
                              bounding box (Sec. 4)                                    */
    double box_margin;     /* bounding box grown by this fraction of its extent, >= 0  */
    int overlap_layers;    /* delta: element layers added to each Omega_p (Sec. 3), >= 0 */
    cgs_precision prec;
    cgs_form form;
    cgs_coarse_solver coarse_solver;  /* 0 (zero-initialised params) = auto        */
    cgs_coarse_operator coarse_operator; /* 0 = cell-wise (Eq. (12))                  */
    int local_cg_steps;    /* 0: exact local solves (explicit A_p^{-1}); k > 0: inexact
                              local solves, k CG steps on each A_p from zero (Sec. 6),
                              one warp per subdomain; needs m_p <= 64 and the FP64 or
                              FP32-bulk form (INVALID_ARG otherwise).  The
                              preconditioner then varies with r, which the flexible
                              PCG and cgs_solve_wrapped's flexible GMRES allow    */
    int fault_negate_subdomain; /* testing aid, 0 in normal use: k > 0 negates the local
                              matrix A_p of subdomain k - 1 (caller numbering) before
                              its inverse is formed, so that the set-up takes its
                              not-SPD path and returns CGS_ERR_NOT_SPD              */
} cgs_params;

typedef struct {
    int64_t nv, ne;        /* vertices, elements                                      */
    int64_t n_free;        /* non-Dirichlet vertices                                  */
    int64_t n_sub;         /* subdomains (max elem_part + 1)                          */
    int64_t n_r;           /* active box vertices (reduced-space unknowns, Sec. 4)    */
    int64_t max_sub_dofs;  /* largest m_p = |R_p|                                     */
    int64_t sum_sub_dofs;  /* sum_p m_p                                               */
    int64_t sum_sub_tri;   /* sum_p m_p (m_p + 1) / 2: entries of the local inverses  */
    size_t footprint_bytes;/* device memory held by the mesh                          */
    double setup_seconds;  /* host wall time of cgs_mesh_setup                        */
    int64_t kernel_launches; /* CUDA kernels this mesh has launched so far           */
    int64_t n_box_entries; /* (vertex, cell) entries of the per-vertex box lists     */
    int64_t n_lane_packs;  /* lane packs of the mixed-form local solves (32 each)    */
    int32_t loop;          /* how solves iterate: 0 host-driven loop, 1 device-side
                              graph loop, 2 persistent cooperative kernel          */
    int32_t coarse_solver; /* the reduced solver in use: CGS_COARSE_DENSE or _XXT   */
    int64_t xxt_nnz;       /* nonzeros of X (XX^T solver), else 0                    */
    int64_t ar_nnz;        /* nonzeros of A_r                                         */
    int32_t coarse_operator; /* the cgs_coarse_operator of the set-up                */
    int64_t n_hyb_entries; /* entries (v, J~_vc, (A J~)_vc) of the hybrid restriction
                              (0 unless the set-up was hybrid)                        */
    int64_t n_jt_entries;  /* entries of the explicit rows of J~ (FP64 form)         */
    int64_t ell_nnz;       /* nonzeros of the assembled free block of A kept for the
                              row applies (0: the element form only)              */
    int64_t ell_slots;     /* its stored entries, padding included (sliced ELL, every
                              row as wide as the widest)                          */
} cgs_mesh_info_t;

/* Launch schedule of a mesh's kernels (cgs_mesh_get_schedule / _set_schedule):
 *   vert_chunk  vertices per block of the vector kernels, multiple of 256 in [256, 8192]
 *   sub_chunk   subdomains per block of the warp-kernel local solves, multiple of 8 in [8, 512]
 *   pack_chunk  lane packs per block of the lane local solves, multiple of 8 in [8, 256]
 *   box_chunk   box-list vertices per interpolation block, multiple of 256 in [256, 4096]
 *   tile_tma    1: element tiles of the mixed-form applies staged by TMA; 0: streamed
 *   persistent  1: mixed-form iterations in one persistent cooperative launch with grid
 *               barriers between the phases; 0 or -1: one launch per phase in the
 *               device-side graph loop (default)
 *   pdl         1: kernels launched with programmatic stream serialization (each may
 *               start while its predecessor drains); 0: ordinary launches
 *   row_packs   1: meshes small enough to have row packs solve each small subdomain
 *               with 4 lanes (full rows; more parallelism); 0: one lane each
 *   interp_cells 1: the interpolation runs over the cell-sorted (vertex, cell)
 *               entries, one warp per cell range, adding into z atomically, and
 *               the PCG dots z.r, z.q follow in their own kernel; 0: by vertex,
 *               the dots fused (fewer launches; the persistent loop always
 *               interpolates by vertex)                                        */
typedef struct {
    int32_t vert_chunk, sub_chunk, pack_chunk, box_chunk, tile_tma, persistent, pdl, row_packs, interp_cells;
} cgs_schedule;

/* Kernel classes reported by the profiler. */
typedef enum {
    CGS_K_APPLY_A64 = 0,   /* outer product q = A p: float64, or float pairs in the
                              mixed forms (also the FP64 inner apply)              */
    CGS_K_APPLY_A32 = 1,   /* s -= A l, float32 inner apply                           */
    CGS_K_LOCAL = 2,       /* local solves                                            */
    CGS_K_RESTRICT = 3,    /* r_r = J~^T s                                            */
    CGS_K_COARSE = 4,      /* u_r = A_r^{-1} r_r                                      */
    CGS_K_INTERP = 5,      /* z += J~ u_r                                             */
    CGS_K_PCG_XR = 6,      /* x, r update and ||r||                                   */
    CGS_K_PCG_DOTS = 7,    /* z.r, z.q (inside CGS_K_INTERP when there is a box space) */
    CGS_K_PCG_P = 8,       /* p = z + beta p                                          */
    CGS_K_OTHER = 9,       /* fills, copies, init, final residual                     */
    CGS_K_LOOP = 10,       /* the persistent loop: whole iterations in one launch     */
    CGS_K_COUNT = 11
} cgs_kernel_class;

/* ---- context --------------------------------------------------------------
 * cgs_create: binds to CUDA device `device`; hbm_budget_bytes caps the sum of
 * footprints of the context's live meshes (0 = no cap).  *ctx owned by the
 * caller until cgs_destroy, which must come after every cgs_mesh_free.      */
cgs_status cgs_create(cgs_ctx** ctx, int device, size_t hbm_budget_bytes);
cgs_status cgs_destroy(cgs_ctx* ctx);
size_t cgs_ctx_bytes_in_use(const cgs_ctx* ctx);

/* ---- setup (Sec. 3 and Sec. 4) ---------------------------------------------
 * Builds everything the solve needs from host arrays, which are copied:
 *   xyz       host, nv*3 float64
 *   conn      host, ne*8 int32, entries in [0, nv)
 *   dirichlet host, nv uint8 (nonzero = homogeneous Dirichlet vertex), or NULL:
 *             every vertex of a boundary face (a face of exactly one element)
 *   elem_part host, ne int32 subdomain id per element (Omega_p), ids in
 *             [0, n_sub); NULL puts every element in one subdomain
 *   params    host; NULL = 4x4x4 boxes, margin 0, delta 1, FP64, hybrid
 * Host work: element matrices (2x2x2 Gauss), Dirichlet set, grown subdomains
 * and the explicit inverses of A_p = R_p A R_p^T (Cholesky, float64), box
 * grid, centroid cells, active box vertices, the reduced operator A_r chosen
 * by params->coarse_operator (cell-wise assembly of Eq. (12), Galerkin
 * J~^T A J~, or vertex-based J^T A J; Sec. 4), and its reduced solver chosen
 * by params->coarse_solver (explicit dense inverse, or the XX^T factor X of
 * Sec. 2 in a nested-dissection order), all in float64; the mixed forms also
 * keep hi/lo float-pair copies of A_r^{-1} or X.  Then one upload to the
 * device.  Synchronous.
 * Errors: INVALID_ARG, INVALID_MESH (index out of range, Jacobian <= 0 at a
 * quadrature point, empty mesh), NOT_SPD, ADMISSION, OOM, CUDA.  On error
 * *out is NULL and nothing stays allocated.                                 */
cgs_status cgs_mesh_setup(cgs_ctx* ctx, const double* xyz, int64_t nv,
                          const int32_t* conn, int64_t ne,
                          const uint8_t* dirichlet, const int32_t* elem_part,
                          const cgs_params* params, cgs_mesh** out);
cgs_status cgs_mesh_free(cgs_mesh* mesh);
cgs_status cgs_mesh_info(const cgs_mesh* mesh, cgs_mesh_info_t* info);
/* Switch the preconditioner form of an existing mesh (no new data needed). */
cgs_status cgs_mesh_set_form(cgs_mesh* mesh, cgs_form form);
/* Host copies of setup results, for checking: dirichlet (nv uint8),
 * box_active (n_r int64 lexicographic box-vertex ids (i + (b_x+1)(j + (b_y+1)k)),
 * sub_ptr (n_sub+1 int64) and sub_idx (sum_sub_dofs int32 ascending vertex ids).
 * Any output pointer may be NULL.  Synchronous.                             */
cgs_status cgs_mesh_export(const cgs_mesh* mesh, uint8_t* dirichlet, int64_t* box_active,
                           int64_t* sub_ptr, int32_t* sub_idx);

/* ---- hot-path steps, device vectors, stream-ordered -------------------------
 * These single-step calls use the mesh's scratch vectors (so they must not
 * overlap each other or a solve on the same mesh).  A bounded device-side wait
 * that expires inside one of them (only the TMA-staged element tiles of the
 * mixed-form applies wait) skips the rest of that call's work and is recorded
 * in the mesh's step status word; cgs_mesh_step_status reports it.
 *
 * cgs_apply_A: y = A x, A = Q^T A_L Q (Sec. 3), float64.  x, y device, nv.  */
cgs_status cgs_apply_A(cgs_mesh* mesh, const double* x, double* y, void* stream);
/* cgs_apply_A_prec: y = A x (Sec. 3) evaluated by one of the mesh's operator
 * kernels, for checking each precision form against its error bound:
 *   CGS_OP_FP64   the float64 operator (as cgs_apply_A);
 *   CGS_OP_INNER  the inner apply of the hybrid step (Eq. (5), s = r - A l):
 *                 x rounded to float32, 28 float32 off-diagonals per element,
 *                 float32 sums, then widened to float64;
 *   CGS_OP_OUTER  the outer operator of the PCG (q = A p): hi/lo float pairs
 *                 (about 48 bits) in the mixed forms.
 * In the FP64 form every op is the float64 operator.  x, y device, nv; Dirichlet
 * entries of x are ignored and y is 0 there.  INVALID_ARG for an unknown op.  */
enum { CGS_OP_FP64 = 0, CGS_OP_INNER = 1, CGS_OP_OUTER = 2 };
cgs_status cgs_apply_A_prec(cgs_mesh* mesh, const double* x, double* y, int op, void* stream);
/* cgs_mesh_step_status: waits for `stream`, then returns CGS_ERR_TIMEOUT if a
 * bounded device wait expired in a single-step call on this mesh (any call of
 * this section and cgs_apply_preconditioner_noalloc) since the last query,
 * else CGS_OK; the status word is reset either way.                          */
cgs_status cgs_mesh_step_status(cgs_mesh* mesh, void* stream);
/* cgs_mesh_set_wait_limits: iteration limits of the bounded device-side waits
 * of this mesh's kernels: tile_wait for the element-tile TMA copies (default
 * 1 << 20 polls) and barrier_wait for the grid barriers of the persistent loop
 * (default 1 << 22 polls).  A testing aid: 0 makes every such wait give up at
 * once, so the timeout path (CGS_ERR_TIMEOUT, the call's work skipped, the
 * context still usable) runs without any fault.  A block that gives up still
 * waits, with its own limit, for the copy it started before it returns.
 * Synchronous.  INVALID_ARG for a negative limit.                            */
cgs_status cgs_mesh_set_wait_limits(cgs_mesh* mesh, int tile_wait, int barrier_wait);
/* cgs_apply_local: l = sum_p R_p^T A_p^{-1} R_p r (Eq. (4)), weighted by
 * W_ov = 1/multiplicity when `weighted` != 0.  Mesh precision.              */
cgs_status cgs_apply_local(cgs_mesh* mesh, const double* r, double* l, int weighted, void* stream);
/* cgs_restrict: r_r = J_L^T Q W s (Sec. 4); s device nv, r_r device n_r.     */
cgs_status cgs_restrict(cgs_mesh* mesh, const double* s, double* rr, void* stream);
/* cgs_coarse_solve: u_r = A_r^{-1} r_r (Sec. 4) by the mesh's reduced solver
 * (dense explicit inverse, or XX^T, Sec. 2); device n_r vectors, float64 in and
 * out.  The FP64 form computes in float64; the mixed forms keep A_r^{-1} (or
 * X) and r_r as hi/lo float pairs (about 48 bits) and multiply on the FP32
 * pipes.                                                                     */
cgs_status cgs_coarse_solve(cgs_mesh* mesh, const double* rr, double* ur, void* stream);
/* cgs_interp: z = W Q^T J_L u_r (Sec. 4); u_r device n_r, z device nv.       */
cgs_status cgs_interp(cgs_mesh* mesh, const double* ur, double* z, void* stream);
/* cgs_apply_preconditioner: z = M r in the mesh's form and precision.       */
cgs_status cgs_apply_preconditioner(cgs_mesh* mesh, const double* r, double* z, void* stream);

/* ---- repeated right-hand sides: projection onto prior solutions -----------
 * For a sequence of solves with the same mesh (a pressure solve per time step),
 * Sec. 5 solves only for the change from the A-orthogonal best fit onto l
 * prior solutions.
 * cgs_mesh_set_projection: keep up to `l` prior solutions of cgs_solve /
 *   cgs_solve_host on this mesh (0 <= l <= CGS_PROJECTION_MAX; 0 = off, the
 *   default).  The kept vectors form an A-orthonormal basis x~_j in float64
 *   (with A x~_j): each solve starts from u_bar = sum_j (x~_j . b) x~_j, runs
 *   the PCG on b - A u_bar with the stopping test still relative to ||b||,
 *   returns u_bar + the correction, then makes the solution A-orthogonal to
 *   the basis and appends it (one extra float64 operator apply; a solution
 *   that adds no direction, below 1e-6 of its A-norm, is not appended); a
 *   full basis restarts from the newest solution.  iters counts the correction's
 *   products A p (0 when the start already meets rtol); relres is
 *   ||b - A x|| / ||b||.  Allocates 2 l nv + 2 nv doubles (freed with the
 *   mesh or by l = 0); resets the basis.  Batches, servers and
 *   cgs_solve_batched do not use it.  INVALID_ARG for l out of range.
 * cgs_mesh_projection_size: the number of kept vectors now.              */
#define CGS_PROJECTION_MAX 64
cgs_status cgs_mesh_set_projection(cgs_mesh* mesh, int l);
cgs_status cgs_mesh_projection_size(const cgs_mesh* mesh, int* k);

/* ---- preconditioner apply without allocation -------------------------------
 * cgs_apply_preconditioner_noalloc: the same z = M r as
 * cgs_apply_preconditioner, for callers that must not allocate device memory
 * at call time: serving loops that forbid allocations after warm-up, and hosts
 * whose device memory is owned by another runtime's pool (an allocation there
 * would bypass that pool's accounting or fail outright).  The call performs no
 * cudaMalloc or cudaFree and uses no allocating library routine.  Its working
 * vectors (z and s in the bulk precision, r_r, u_r and the XX^T pass's t)
 * live in one static
 * device array of CGS_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library keeps until the process exits.
 *   limits  mesh nv <= CGS_NOALLOC_MAX_NV and n_r <= CGS_NOALLOC_MAX_NR, else
 *           CGS_ERR_INVALID_ARG with a message naming the limit.
 *   set-up  the first call on a device looks up the array's device address
 *           (cudaGetSymbolAddress) with that device current; make that first
 *           call before any stream capture.
 *   sharing every call on a device uses the same array, which keeps the
 *           previous call's contents (the call clears what must start at 0).
 *           Calls that overlap on the GPU (other streams, other threads, or
 *           another mesh) race on it: serialise them.
 *   status  an expired element-tile wait is recorded in the mesh's step
 *           status word (cgs_mesh_step_status), which setup allocated.
 * r, z device vectors of length nv; stream-ordered.  The paper has no
 * counterpart.                                                              */
#define CGS_NOALLOC_MAX_NV 131072
#define CGS_NOALLOC_MAX_NR 8192
#define CGS_NOALLOC_SCRATCH_BYTES ((size_t)16 * CGS_NOALLOC_MAX_NV + (size_t)24 * CGS_NOALLOC_MAX_NR)
cgs_status cgs_apply_preconditioner_noalloc(cgs_mesh* mesh, const double* r, double* z, void* stream);

/* ---- solve ----------------------------------------------------------------
 * cgs_solve: flexible PCG (Polak-Ribiere beta, x0 = 0) on A x = b for nrhs
 * right-hand sides stored back to back (b[k*nv ...]); stops when the
 * recursive residual satisfies ||r|| <= rtol ||b|| or after maxit products
 * A p.  b, x device.  iters[k] = products A p used, relres[k] = true
 * ||b - A x|| / ||b|| (0 when b = 0), both host arrays of nrhs, always
 * written.  Synchronous (waits for the stream).  Returns NO_CONVERGENCE or
 * BREAKDOWN for the first right-hand side that failed; the others are still
 * solved.                                                                   */
cgs_status cgs_solve(cgs_mesh* mesh, const double* b, double* x, int nrhs, double rtol,
                     int maxit, int* iters, double* relres, void* stream);
/* cgs_solve_host: as cgs_solve with b and x in HOST memory; copies them to
 * and from the device inside the call (pinned memory makes this faster).    */
cgs_status cgs_solve_host(cgs_mesh* mesh, const double* b_host, double* x_host, int nrhs,
                          double rtol, int maxit, int* iters, double* relres, void* stream);

/* ---- other outer iterations around the same preconditioner -----------------
 * cgs_solve_wrapped: A x = b for one right-hand side with
 *   CGS_METHOD_PCG         the flexible PCG of cgs_solve (restart ignored);
 *   CGS_METHOD_RICHARDSON  Schwarz-Richardson, x += M (b - A x) from x = 0, the
 *                          paper's alternative wrapper (Sec. 3); iters counts the
 *                          updates of x;
 *   CGS_METHOD_FGMRES      flexible GMRES(restart), right-preconditioned, x = 0
 *                          first: the Arnoldi basis V of the residual space and the
 *                          preconditioned directions Z = M V are kept, so M may vary
 *                          between steps (inexact local solves, Sec. 6); the
 *                          Hessenberg least-squares problem is solved by Givens
 *                          rotations on the host; iters counts the products A z.
 * M is the mesh's preconditioner (form and precision); vectors and
 * arithmetic of the outer iteration are float64 on the device.  Stops when the
 * residual norm (true for Richardson and at every GMRES restart, the
 * least-squares estimate inside a cycle) is <= rtol ||b||.  b, x device
 * vectors of length nv; iters and relres (the last residual norm / ||b||)
 * host scalars, always written.  Synchronous; allocates (restart + 1 +
 * restart) nv doubles for GMRES, 3 nv for Richardson, freed before it
 * returns.  Returns NO_CONVERGENCE after maxit, BREAKDOWN on a non-finite
 * value, TIMEOUT when a bounded device wait expired, INVALID_ARG for an
 * unknown method or restart outside [1, 1024].                              */
typedef enum { CGS_METHOD_PCG = 0, CGS_METHOD_RICHARDSON = 1, CGS_METHOD_FGMRES = 2 } cgs_method;
cgs_status cgs_solve_wrapped(cgs_mesh* mesh, const double* b, double* x, cgs_method method, double rtol, int maxit,
                             int restart, int* iters, double* relres, void* stream);

/* ---- profiling --------------------------------------------------------------
 * cgs_profile_enable: when on, every kernel the mesh launches is bracketed by
 * CUDA events recorded on its launching stream (adds host cost per launch).
 * cgs_profile_read: waits for the device, then writes per kernel class the
 * summed event time in milliseconds (ms[CGS_K_COUNT]) and the launch count
 * (launches[CGS_K_COUNT]) since the last read, and resets them.            */
cgs_status cgs_profile_enable(cgs_mesh* mesh, int enable);
cgs_status cgs_profile_read(cgs_mesh* mesh, double* ms, int64_t* launches);

/* ---- batches: many meshes and right-hand sides in each launch ---------------
 * cgs_batch_create: a solve plan over `nmesh` meshes (same context, same
 * precision and form) with `nrhs` right-hand sides each, i.e. nmesh*nrhs
 * slots numbered slot = mesh_index * nrhs + rhs.  Every kernel of the
 * iteration covers all slots in one launch; slots stop independently (each
 * has its own scalars and stopping test) and the device-side loop ends when
 * the last slot stops.  The batch holds its own vector pools (the meshes'
 * data is shared, not copied) and must be freed before its meshes.
 * cgs_batch_solve: b[slot], x[slot] are device vectors of the slot's mesh
 * (host arrays of nmesh*nrhs device pointers); iters, relres (and status
 * when not NULL) are host arrays of nmesh*nrhs, always written.  Synchronous.
 * Returns the first slot's error if any slot failed.
 * cgs_solve_batched: create + solve + free in one call.                     */
typedef struct cgs_batch cgs_batch;
cgs_status cgs_batch_create(cgs_ctx* ctx, cgs_mesh* const* meshes, int nmesh, int nrhs, cgs_batch** out);
cgs_status cgs_batch_free(cgs_batch* batch);
cgs_status cgs_batch_solve(cgs_batch* batch, const double* const* b, double* const* x, double rtol, int maxit,
                           int* iters, double* relres, int* status, void* stream);
int64_t cgs_batch_launches(const cgs_batch* batch);
/* Autotuner: time the local solves over subdomain chunks {8,16,32,64}, the
 * vector kernels over vertex chunks {256,...,2048}, the interpolation over
 * box-list chunks {256, 512, 1024} and, in the mixed forms, the tiled
 * operator applies with TMA-staged or thread-streamed element tiles, on the
 * object's own data; keep the fastest schedule (rebuilds the work tables and
 * the loop graph).
 * Synchronous; call between solves.  Setup picks a default schedule that
 * gives about four blocks per SM.                                          */
cgs_status cgs_mesh_tune(cgs_mesh* mesh, void* stream);
/* The schedule in use, and an explicit one (INVALID_ARG if a field is out of
 * range; synchronous, call between solves).                                */
cgs_status cgs_mesh_get_schedule(const cgs_mesh* mesh, cgs_schedule* out);
cgs_status cgs_mesh_set_schedule(cgs_mesh* mesh, const cgs_schedule* schedule);
cgs_status cgs_batch_tune(cgs_batch* batch, void* stream);
cgs_status cgs_solve_batched(cgs_mesh* const* meshes, int nmesh, const double* const* b, double* const* x,
                             int nrhs, double rtol, int maxit, int* iters, double* relres, void* stream);

/* ---- serving: continuous batching --------------------------------------------
 * A server keeps up to `max_slots` solves in flight, all in one precision and
 * form, each solved to rtol within maxit products.  Meshes stay set up
 * (resident) across requests; the caller keeps them alive while requests on
 * them are pending.
 *
 * Admission is by device-memory footprint.  The working vectors of every
 * running solve live in one arena of `pool_nv` vertex entries and `pool_nr`
 * reduced (box) entries, allocated at creation.  A request needs nv vertex
 * entries (56 bytes each in the FP64 form, 48 in the mixed forms), n_r reduced
 * entries and a few partial-sum entries; it is admitted, in arrival order,
 * when a slot is free and the arena has room for all three (first fit).  A
 * request that waits blocks those behind it (no overtaking), so large
 * requests are not starved.
 *
 * cgs_server_create: pool_nv >= 1, pool_nr >= 0.  ADMISSION if the arena
 *   exceeds the context's HBM budget.
 * cgs_submit: queue one solve; b and x are device vectors of the mesh that
 *   the caller keeps valid until cgs_poll reports done.  ADMISSION if the
 *   request could never fit the arena.  Host-only, returns at once.
 * cgs_server_step: admits queued requests (starting their iteration), runs
 *   `iterations` PCG iterations over every running slot in shared launches
 *   (slots at different iteration counts), then retires the slots that
 *   stopped: true residual, solution copied to x, arena space released.
 *   Synchronous.  active/queued/finished (each may be NULL) report counts.
 * cgs_poll: done = 1 once the request has finished (then iters, relres and
 *   status are its results and the ticket is released).
 * cgs_server_drain: copies up to `cap` requests finished since the last
 *   drain (ticket and, where the arrays are not NULL, iters, relres, status)
 *   and releases their tickets; returns how many, or -1 on a bad argument.
 *   A ticket already released by cgs_poll is skipped.
 * cgs_server_footprint: arena bytes a request on `mesh` would hold.
 * cgs_server_stats: arena capacity and bytes held by running solves.       */
typedef struct cgs_server cgs_server;
cgs_status cgs_server_create(cgs_ctx* ctx, int max_slots, int64_t pool_nv, int64_t pool_nr, cgs_precision prec,
                             cgs_form form, double rtol, int maxit, cgs_server** out);
cgs_status cgs_server_free(cgs_server* server);
cgs_status cgs_submit(cgs_server* server, cgs_mesh* mesh, const double* b, double* x, uint64_t* ticket);
cgs_status cgs_server_step(cgs_server* server, int iterations, void* stream, int* active, int* queued,
                           int* finished);
cgs_status cgs_poll(cgs_server* server, uint64_t ticket, int* done, int* iters, double* relres, int* status);
int cgs_server_drain(cgs_server* server, uint64_t* tickets, int* iters, double* relres, int* status, int cap);
cgs_status cgs_server_footprint(const cgs_server* server, const cgs_mesh* mesh, size_t* bytes);
cgs_status cgs_server_stats(const cgs_server* server, size_t* arena_bytes, size_t* bytes_in_use, int* active,
                            int* queued);
int64_t cgs_server_launches(const cgs_server* server);

/* ---- p-multigrid wrap: spectral-element levels around the coarse solve ----
 * The coarse-grid solve is the N = 1 level of a p-multigrid preconditioner
 * for the spectral-element (SEM) Poisson problem of order N (Sec. 1, Sec. 5).
 * A cgs_pmg holds the SEM levels of orders N_0 > N_1 > ... > 1 on the
 * hexahedral mesh of a cgs_mesh, and applies the preconditioner of Eq. (13),
 * additive between levels,
 *     z = M_{N0}^-1 r + J_1 (M_{N1}^-1 r_1 + J_2 (... + J_c M_c J_c^T ...)),
 * r_{l+1} = J_{l+1}^T r_l, where
 *   - M_N^-1 = W_N sum_e R_{N,e}^T A~_{N,e}^-1 R_{N,e} (Eq. (14)) is the
 *     element-local additive Schwarz smoother: R_{N,e} takes the element's
 *     own (N+1)^3 nodes, A~ is the separable approximation of the element
 *     problem solved by fast diagonalisation, W_N = 1 / (elements holding
 *     the node);
 *   - J from an order to the next finer one is element-wise tensor-product
 *     Lagrange interpolation between the GLL nodes, averaged over the copies
 *     of each fine node (J = W_f Q_f^T I Q_c), and J^T its transpose;
 *   - M_c, at order 1, is ONE application of the mesh's two-level Schwarz
 *     preconditioner (cgs_apply_preconditioner, in the mesh's form and
 *     precision): inside a Krylov method the coarse problem needs no exact
 *     solve (Sec. 3, opening paragraph).
 * The SEM operator of order N is A_N = Q^T A_L Q with A^e = Dhat^T G^e Dhat,
 * GLL quadrature at the nodes and the trilinear map of each hexahedron; every
 * node of a boundary face is Dirichlet.  Precision follows the mesh: all
 * float64 under an FP64 mesh; under the mixed forms the operator runs in
 * float-pair arithmetic (about 48 bits) and the smoothers and transfers in
 * float (vectors of the API and GMRES stay float64).
 *
 * Levels are numbered 0 (order orders[0]) to n_orders (order 1, whose nodes
 * are the mesh vertices in the mesh's own numbering).  Vectors of level l are
 * float64 DEVICE arrays over its global nodes; Dirichlet entries are ignored
 * on input and written 0 on output.  The global numbering of level l < n_orders
 * starts with the mesh vertices, then the nodes inside edges, faces and
 * elements; cgs_pmg_node_map gives it per element.
 *
 * cgs_pmg_setup: `mesh` must have the default Dirichlet set (boundary-face
 *   vertices) and must outlive the cgs_pmg; xyz (nv*3) and conn (ne*8,
 *   lexicographic vertex order) are the HOST arrays the mesh was set up
 *   from (checked against its sizes; copied).  orders: n_orders (1..4) values,
 *   strictly decreasing, each in [2, 8] (e.g. {7, 3} for 7 -> 3 -> 1).
 *   Device memory per element at order N (p = N + 1): 6 p^3 doubles of
 *   geometric factors, p^3 int32 node numbers and 3 p (p + 1) doubles of
 *   smoother factors, plus about four doubles per global node; it is not
 *   counted against the context's budget.  INVALID_ARG on a bad argument, INVALID_MESH on a
 *   non-positive Jacobian at a GLL node, OOM.  Synchronous.
 * cgs_pmg_info: order, global nodes and free (non-Dirichlet) nodes of a level.
 * cgs_pmg_node_map: HOST array of ne*(N+1)^3 global node numbers, element by
 *   element, local node (i, j, k) at i + (N+1)(j + (N+1) k); for level
 *   n_orders this is conn.
 * cgs_pmg_node_coords: HOST array of n_nodes*3 node coordinates.
 * cgs_pmg_apply_A: y = A_N x on level l < n_orders.
 * cgs_pmg_smooth: z = M_N^-1 r (Eq. (14)) on level l < n_orders.
 * cgs_pmg_restrict: rc = J^T rf from level l to level l + 1.
 * cgs_pmg_prolong: uf = J uc from level l + 1 to level l.
 * cgs_pmg_apply_preconditioner: z = M r of Eq. (13) on level 0.
 * cgs_pmg_solve: A_{N0} x = b on level 0 by flexible GMRES(restart) with
 *   that preconditioner (Sec. 5: GMRES on the pressure, p-multigrid
 *   preconditioned), x = 0 first, stopping at ||b - A x|| <= rtol ||b||
 *   (the least-squares estimate inside a cycle, the true residual at every
 *   restart); iters = products A z, relres as in cgs_solve_wrapped.
 *   Synchronous.  The first solve, and one with a larger restart than any
 *   before, allocates the GMRES workspace (about 2 restart + 3 vectors of
 *   level 0), which the cgs_pmg keeps until cgs_pmg_free.
 *   NO_CONVERGENCE after maxit, BREAKDOWN on a non-finite value, TIMEOUT
 *   when a bounded device wait of the coarse preconditioner expired.
 * The single-step calls are asynchronous on `stream` and use work vectors of
 * the cgs_pmg (calls on one cgs_pmg must not overlap).                     */
typedef struct cgs_pmg cgs_pmg;
cgs_status cgs_pmg_setup(cgs_mesh* mesh, const double* xyz, int64_t nv, const int32_t* conn, int64_t ne,
                         const int32_t* orders, int n_orders, cgs_pmg** out);
cgs_status cgs_pmg_free(cgs_pmg* pmg);
cgs_status cgs_pmg_info(const cgs_pmg* pmg, int level, int* order, int64_t* n_nodes, int64_t* n_free);
cgs_status cgs_pmg_node_map(const cgs_pmg* pmg, int level, int32_t* l2g);
cgs_status cgs_pmg_node_coords(const cgs_pmg* pmg, int level, double* xyz);
cgs_status cgs_pmg_apply_A(cgs_pmg* pmg, int level, const double* x, double* y, void* stream);
cgs_status cgs_pmg_smooth(cgs_pmg* pmg, int level, const double* r, double* z, void* stream);
cgs_status cgs_pmg_restrict(cgs_pmg* pmg, int level, const double* rf, double* rc, void* stream);
cgs_status cgs_pmg_prolong(cgs_pmg* pmg, int level, const double* uc, double* uf, void* stream);
cgs_status cgs_pmg_apply_preconditioner(cgs_pmg* pmg, const double* r, double* z, void* stream);
cgs_status cgs_pmg_solve(cgs_pmg* pmg, const double* b, double* x, double rtol, int maxit, int restart,
                         int* iters, double* relres, void* stream);

const char* cgs_status_string(cgs_status s);
const char* cgs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CGS_H */
