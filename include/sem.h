/*
 * sem.h -- C ABI of the GB300 spectral-element pressure-Poisson library.
 *
 * The library solves the pressure-Poisson problem of a semi-implicit spectral
 * element (SEM) Navier-Stokes step (Fischer et al., "Highly Optimized
 * Full-Core Reactor Simulations on Summit", Sec. 2-3) on one GPU:
 * matrix-free tensor-product stiffness operator on deformed hexahedra, direct
 * stiffness summation (gather-scatter), p-multigrid preconditioning with
 * Chebyshev-accelerated Jacobi smoothing, Jacobi-PCG and flexible CG.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Mesh: a box of ex*ey*ez hexahedra on a vertex lattice of
 *   (ex+1)(ey+1)(ez+1) points, each element mapped trilinearly from [-1,1]^3
 *   (the isoparametric map of Sec. 2 with straight edges).  Element
 *   e = ix + ex*(iy + ey*iz).
 * - Fields are "E-layout" vectors: E*(N+1)^3 values, element-major, point
 *   (i,j,k) of an element at i + (N+1)*(j + (N+1)*k), i along r (Sec. 2, Eq. 2:
 *   nodal values u^e_ijk on Gauss-Lobatto-Legendre points).  A field is
 *   "continuous" when all local copies of a shared node hold the same value.
 * - Vectors passed to the library are caller-owned DEVICE memory unless the
 *   entry point says HOST.  The library never frees them.  The library owns
 *   everything reachable from a handle (geometry, numbering, workspaces) and
 *   frees it in the matching *_destroy.
 * - All device work is enqueued on the caller's CUDA stream (`stream`, a
 *   cudaStream_t passed as void*; NULL = the legacy default stream).  Entry
 *   points that return values to the host synchronise that stream.
 * - Every entry point returns a sem_status; on failure sem_last_error() holds a
 *   message (thread-local) and outputs are unspecified.  No C++ exception
 *   crosses this boundary.  Arguments are validated before any device work.
 * - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SEM_OK = 0,
  SEM_EINVAL = 1,    /* bad argument, size, null pointer, folded element */
  SEM_ENOMEM = 2,    /* device or host allocation failed */
  SEM_ECUDA = 3,     /* a CUDA runtime call failed */
  SEM_ENOTCONV = 4,  /* solver hit max_iter before the tolerance */
  SEM_ENUMERIC = 5,  /* NaN or Inf met in a solver */
  SEM_EAGAIN = 6,    /* request still pending (sem_poll) */
  SEM_EBUSY = 7,     /* no free slot or memory for a request (sem_submit) */
  SEM_ETIMEOUT = 8   /* a bounded wait inside a kernel ran out (reported by
                        the solves, sem_pmg_vcycle and the staged kinds of
                        sem_ax; see sem_solve) */
} sem_status;

typedef enum { SEM_F64 = 0, SEM_F32 = 1, SEM_F16 = 2, SEM_BF16 = 3 } sem_dtype;

enum { SEM_DIRICHLET = 0, SEM_NEUMANN = 1 };
enum { SEM_GEOM_STORED = 0, SEM_GEOM_TRILINEAR = 1 };
/* How FP64 operator applications are computed (results agree to ~1e-14):
 * SEM_ARITH_PAIR   FP32-pair ("double-float") arithmetic on the FP32 pipes,
 *                  geometric factors stored as hi/lo float pairs (default).
 *                  It covers the FP32 exponent range: input values, factors
 *                  and partial sums of magnitude about 1e-38 to 3e38 keep
 *                  FP64-level relative accuracy; values outside it are
 *                  taken as zero.  Scale the data into that range or use
 * SEM_ARITH_NATIVE native FP64 instructions, factors stored as doubles.
 * Recomputed (trilinear) geometry always uses native FP64. */
enum { SEM_ARITH_PAIR = 0, SEM_ARITH_NATIVE = 1 };

typedef struct sem_mesh sem_mesh;
typedef struct sem_pmg sem_pmg;

/* Mesh description.  verts (HOST, may be NULL): vertex lattice
 * [(ex+1)(ey+1)(ez+1)][3], vertex (a,b,c) at a + (ex+1)(b + (ey+1)c); it is
 * copied during sem_mesh_create.  When NULL the library builds the unit-cube
 * lattice and moves every vertex strictly inside the cube by
 * (2u-1)*jitter/(ex,ey,ez) per coordinate, u = top 53 bits of
 * splitmix64(seed + (3*vertex + coordinate + 1) * 0x9E3779B97F4A7C15) * 2^-53.
 * bc: SEM_DIRICHLET (u = 0 on the box boundary) or SEM_NEUMANN.
 * geom: SEM_GEOM_STORED keeps the six geometric factors per point in HBM;
 * SEM_GEOM_TRILINEAR keeps only the 8 vertices per element and recomputes
 * the factors inside the operator kernel. */
typedef struct {
  int32_t ex, ey, ez;  /* elements per direction, each >= 1 */
  int32_t N;           /* polynomial order, 1 <= N <= SEM_MAX_ORDER */
  double jitter;       /* built-in generator only */
  uint64_t seed;       /* built-in generator only */
  int32_t bc;
  int32_t geom;
  const double *verts;
  int32_t f64_arith;   /* SEM_ARITH_PAIR or SEM_ARITH_NATIVE */
} sem_mesh_desc;

#define SEM_MAX_ORDER 11

/* Build the mesh, its geometric factors (Sec. 2: isoparametric map, six
 * symmetric factors G = w det(J) J^-1 J^-T per GLL point, mass B = w det(J)),
 * the shared-node numbering for gather-scatter (Sec. 3: global vertex ids)
 * and the Jacobi diagonal.  Synchronises `stream`.
 * Errors: SEM_EINVAL (sizes, order, det(J) <= 0, more than 2^31-1 local
 * points), SEM_ENOMEM, SEM_ECUDA. */
sem_status sem_mesh_create(const sem_mesh_desc *desc, void *stream, sem_mesh **out);
sem_status sem_mesh_destroy(sem_mesh *mesh);

/* Test hook (host-side fault injection): after > 0 makes the after-th
 * device allocation of the library from now on fail with SEM_ENOMEM before
 * it reaches the CUDA allocator (the call that allocates returns SEM_ENOMEM
 * and frees what it had built); 0 disarms.  Process-wide.
 * Errors: SEM_EINVAL (after < 0). */
sem_status sem_inject_alloc_failure(int32_t after);

/* Test hook: sets the fine level's wait-error flag from the host, as a
 * kernel whose bounded wait ran out would, so that the next call that reads
 * the flags (a solve, sem_pmg_vcycle, a staged kind of sem_ax) reports
 * SEM_ETIMEOUT and clears it.  Nothing runs on the device.
 * Synchronises `stream`.  Errors: SEM_EINVAL (null mesh), SEM_ECUDA. */
sem_status sem_inject_wait_error(sem_mesh *mesh, void *stream);

/* n_local = E (N+1)^3, n_global = (ex N+1)(ey N+1)(ez N+1) unique nodes,
 * dev_bytes = device memory owned by the mesh.  Any output may be NULL. */
sem_status sem_mesh_info(const sem_mesh *mesh, int64_t *n_local, int64_t *n_global,
                         size_t *dev_bytes);

enum {
  SEM_FIELD_X = 0, SEM_FIELD_Y = 1, SEM_FIELD_Z = 2, /* physical coordinates */
  SEM_FIELD_MASS = 3,  /* B = w_i w_j w_k det(J), unassembled */
  SEM_FIELD_MULT = 4,  /* number of local copies of each node */
  SEM_FIELD_MASK = 5,  /* 0 on Dirichlet boundary nodes, else 1 */
  SEM_FIELD_DINV = 6   /* mask / assembled diagonal of A (Jacobi) */
};
/* Write one per-point field of the mesh, FP64 E-layout, into out (device,
 * n_local doubles). */
sem_status sem_mesh_field(sem_mesh *mesh, int32_t which, double *out, void *stream);

enum { SEM_AX_LOCAL = 0, SEM_AX_ASSEMBLED = 1 };
/* Stiffness operator (Sec. 2, footnote 1: u_r = Dhat u along each direction,
 * then w = sum_d Dhat_d^T sum_e G_de u_e).
 * SEM_AX_LOCAL:     w = A_L u, element by element (no summation).
 * SEM_AX_ASSEMBLED: w = mask * gs(A_L u).
 * dtype: SEM_F64 (u, w double) or SEM_F32 (u, w float; factors rounded to
 * float once at mesh creation), or SEM_F16 / SEM_BF16: u, w float and FP32
 * arithmetic, but the six factors stored in 16 bits, G ~= scale_ef * q_p with
 * scale_ef = float(max_p |G_ef,p|) per element e and factor f and q_p = G_p /
 * scale_ef rounded once from FP64 (nearest, ties to even).  The 16-bit copy is
 * built (and kept) on the first such call; this synchronises once.  u and w
 * are E-layout device vectors of n_local elements and must not overlap; for
 * the 32- and 16-bit kinds on stored geometry u must be 16-byte aligned
 * (SEM_EINVAL otherwise).  The assembled FP32 forms sum the copies of a node
 * across x-, then y-, then z-faces: every copy receives the same bits.
 * The 32- and 16-bit kinds on stored geometry stage their inputs by bulk
 * copies with bounded waits: those calls synchronise `stream`, read the
 * mesh's wait flag and return SEM_ETIMEOUT (w incomplete) if a wait ran out
 * (the flag is cleared). */
sem_status sem_ax(sem_mesh *mesh, sem_dtype dtype, const void *u, void *w, int32_t flags,
                  void *stream);

/* Direct stiffness summation in place (Sec. 2: C0 continuity; Sec. 3: gs):
 * every local copy of a node receives the sum over its copies, summed across
 * x-, then y-, then z-faces (a pairwise tree; no Dirichlet mask).  All copies
 * end bit-identical.  dtype SEM_F64 or SEM_F32. */
sem_status sem_gs(sem_mesh *mesh, sem_dtype dtype, void *u, void *stream);

/* Inner product over unique nodes of two FP64 E-layout vectors,
 * sum_l u_l v_l / mult_l (equal to the Euclidean product of the unique values
 * when u and v are continuous).  Writes *result (HOST); synchronises. */
sem_status sem_dot(sem_mesh *mesh, const double *u, const double *v, double *result,
                   void *stream);

/* The inner product of sem_dot for callers that cannot let the library
 * allocate device memory (a fixed device-memory budget, or a loop that must
 * not pay for the device synchronisation of cudaMalloc/cudaFree).  The paper
 * has no counterpart; this is a service of the library.  The reduction
 * scratch (64 KiB: one partial per CTA of 8192 points plus a counter) is a
 * static device array that every GPU which loads the library keeps until the
 * process exits; nothing is allocated per call.  result is DEVICE memory (one
 * double); the call does not synchronise the stream.  Meshes of more than
 * 67,092,480 local points return SEM_EINVAL (use sem_dot).  The first call on
 * a device looks up the scratch address; make it before any stream capture.
 * All calls share the one scratch array, so calls whose kernels may overlap
 * on the GPU (different streams without ordering) race and must not be
 * issued. */
sem_status sem_dot_noalloc(const sem_mesh *mesh, const double *u, const double *v,
                           double *result, void *stream);

/* p-multigrid description (Sec. 3, pMG: levels of decreasing order, tensor
 * interpolation between them, Chebyshev-accelerated point-Jacobi smoothing,
 * preconditioner arithmetic optionally in 32-bit). */
typedef struct {
  int32_t nlevels;          /* 1..8; orders[0] must equal the mesh order */
  int32_t orders[8];        /* strictly decreasing, e.g. {7, 3, 1} */
  int32_t cheb_degree;      /* Chebyshev degree per smoothing, >= 1 */
  int32_t lanczos_steps;    /* steps of the lambda_max estimate, >= 2 */
  uint64_t seed;            /* start vector of the lambda_max estimate */
  int32_t smoother_dtype;   /* sem_dtype of the smoothed levels: F64, F32, or
                               F16 / BF16 (FP32 vectors and arithmetic,
                               factors stored as in sem_ax) */
  double coarse_tol;        /* coarsest level: FP64 Jacobi-PCG relative tol */
  int32_t coarse_maxit;     /* ... and iteration cap (tol <= 0: exactly maxit) */
  int32_t coarse_mode;      /* SEM_COARSE_JACOBI or SEM_COARSE_MG (below) */
  int32_t smoother;         /* SEM_SMOOTH_JACOBI, SEM_SMOOTH_ASM,
                               SEM_SMOOTH_ASM_TC or SEM_SMOOTH_ASM_TF32 (below) */
  int32_t coarse_ctas;      /* CTAs of the persistent N = 1 coarse kernel: 0 =
                               one per SM (capped by the lattice size), k > 0 =
                               at most k.  Small caps let the coarse solves of
                               many problems run side by side (sem_batch);
                               the CTA count fixes the order of the coarse
                               solver's reductions, so results are identical
                               only between equal caps. */
} sem_pmg_desc;

/* Smoother of the smoothed levels, Chebyshev-accelerated in both cases (Sec. 3).
 * SEM_SMOOTH_JACOBI: point Jacobi.
 * SEM_SMOOTH_ASM: overlapping additive Schwarz (Sec. 3, Eq. 3): every element
 * extended by one point into each face neighbour, a separable local operator
 * (1D SEM stiffness and mass assembled over the neighbour, the element and the
 * other neighbour at their mean lengths) inverted by fast diagonalisation,
 * face data only, contributions summed.  Orders up to N = 9.
 * SEM_SMOOTH_ASM_TC: the same smoother with the FP32 local solves on the
 * tensor cores (each directional transform of an extended element one
 * 128 x 16 x 16 TF32 product, FP32 accuracy from a head + remainder split of
 * both operands) for orders up to N = 8 (at N = 9 the 144 pencils exceed the
 * 128 accumulator rows and that level's local solves stay on the CUDA cores);
 * FP32 smoothing only (smoother_dtype F32, F16 or BF16, else SEM_EINVAL).
 * SEM_SMOOTH_ASM_TF32: as SEM_SMOOTH_ASM_TC without the remainder split: the
 * operands of the local solves are rounded to TF32 (11 significant bits), so
 * the smoother is that accurate; half the shared memory per element. */
enum { SEM_SMOOTH_JACOBI = 0, SEM_SMOOTH_ASM = 1, SEM_SMOOTH_ASM_TC = 2, SEM_SMOOTH_ASM_TF32 = 3 };

/* Coarsest-level solver (the coarsest order must be 1 for SEM_COARSE_MG).
 * SEM_COARSE_JACOBI: FP64 Jacobi-PCG (the default).
 * SEM_COARSE_MG: FP64 flexible CG preconditioned by one geometric multigrid
 * V(2,2) cycle on the N = 1 vertex lattice (Galerkin 27-point operators,
 * Chebyshev-Jacobi smoothing, dense bottom solve); same tolerance and cap.
 * The paper solves its coarse grid with algebraic multigrid (Sec. 4). */
enum { SEM_COARSE_JACOBI = 0, SEM_COARSE_MG = 1 };

/* Build the hierarchy on the mesh's vertices and boundary condition.
 * Chebyshev interval per smoothed level: [lambda_hi/10, lambda_hi] with
 * lambda_hi = 1.1 * (Lanczos estimate of lambda_max(D^-1 A)).
 * The pMG handle refers to the mesh, which must outlive it.  Synchronises. */
sem_status sem_pmg_setup(sem_mesh *mesh, const sem_pmg_desc *desc, void *stream,
                         sem_pmg **out);
sem_status sem_pmg_destroy(sem_pmg *pmg);
/* Chebyshev interval of level l (HOST outputs). */
sem_status sem_pmg_info(const sem_pmg *pmg, int32_t level, double *lam_lo, double *lam_hi);
/* Iterations the coarsest-level solver took in the last V-cycle (HOST
 * output; synchronises the stream the V-cycle ran on). */
sem_status sem_pmg_coarse_iters(const sem_pmg *pmg, void *stream, int32_t *iters);
/* The solve of the coarsest level alone, as a V-cycle runs it (Sec. 4: the
 * coarse-grid solve): b is a right-hand side of that level (FP64 E-layout
 * device vector of E (N_c+1)^3 values, assembled; masked under Dirichlet),
 * x receives the solution after the coarse solver's tolerance or iteration
 * cap (sem_pmg_desc coarse_tol, coarse_maxit, coarse_mode).  Does not
 * synchronise. */
sem_status sem_pmg_coarse_solve(sem_pmg *pmg, const double *b, double *x, void *stream);
/* One V-cycle z = M r on the finest level (FP64 E-layout device vectors).
 * Synchronises `stream` to read the levels' wait flags: SEM_ETIMEOUT (z
 * incomplete; flags cleared) if a bounded wait in a smoother kernel ran
 * out. */
sem_status sem_pmg_vcycle(sem_pmg *pmg, const double *r, double *z, void *stream);

enum { SEM_SOLVER_PCG = 0, SEM_SOLVER_FLEXCG = 1, SEM_SOLVER_FGMRES = 2 };
typedef struct {
  int32_t solver;    /* SEM_SOLVER_PCG (Jacobi, Sec. 3), SEM_SOLVER_FLEXCG, or
                        SEM_SOLVER_FGMRES (Sec. 3: flexible GMRES, classical
                        Gram-Schmidt; pMG preconditioner, or Jacobi when pmg is
                        NULL) */
  double tol;        /* stop when ||r|| <= tol ||b|| (unique-dof 2-norm) */
  int32_t max_iter;
  int32_t check_every; /* read the residual norm every k iterations (>= 1; CG forms) */
  int32_t restart;   /* FGMRES: Krylov vectors per cycle, 1..32 (0: 20) */
  int32_t use_graph; /* FlexCG only: 1 runs iterations 2.. as one CUDA graph
                        launch (a device-side while loop whose stopping test
                        runs on the GPU; the host reads the result once), 0
                        the host-driven loop.  Results are identical; the
                        graph saves the per-launch host cost on small
                        problems.  check_every is ignored (the test runs
                        every iteration).  The mesh keeps one graph, captured
                        again when the pMG or x changes. */
  int32_t zero_guess; /* 1: start from x = 0 and ignore x's input (x is output
                         only: sem_solve_host copies nothing to x's device
                         copy, and no operator is applied to the guess); 0:
                         x holds the initial guess.  The results equal those
                         of a zero-filled x bit for bit. */
} sem_solve_desc;

typedef struct {
  int32_t iters;
  int32_t status;      /* sem_status of the solve */
  double res0, res;    /* initial and final residual norms */
  double bnorm;
  double time_ms;      /* device time of the solve (CUDA events) */
} sem_solve_info;

/* Solve A x = b (FP64 outer iteration).  b: assembled right-hand side
 * (continuous, masked under Dirichlet; mean-free under Neumann: SEM_EINVAL if
 * |sum b / mult| > 1e-10 * ||b||_1 / mult).  x: initial guess in, solution
 * out.  pmg: NULL for Jacobi-PCG; required for SEM_SOLVER_FLEXCG; optional
 * for SEM_SOLVER_FGMRES.  FGMRES keeps 2 restart + 1 FP64 vectors of n_local
 * (allocated on first use, kept by the mesh); its residual test uses the
 * least-squares residual of each step and, at the end of a cycle, the
 * residual recomputed from x.
 * Returns SEM_OK, SEM_ENOTCONV (max_iter reached; x and info hold the last
 * iterate), SEM_ENUMERIC (NaN/Inf) or SEM_ETIMEOUT: a kernel's bounded wait
 * (a bulk copy that did not complete within its poll limit) ran out during
 * the solve or since the last solve on this mesh, that kernel left its work
 * undone, and x is not to be trusted.  The flags behind SEM_ETIMEOUT are
 * read and cleared at the end of every solve (sem_solve, sem_solve_host,
 * sem_solve_projected, served requests).  Synchronises. */
sem_status sem_solve(sem_mesh *mesh, sem_pmg *pmg, const double *b, double *x,
                     const sem_solve_desc *desc, sem_solve_info *info, void *stream);

/* As sem_solve with b and x in HOST memory: copies b (and the guess x) to the
 * device, solves, copies x back.  Device vectors are owned by the mesh. */
sem_status sem_solve_host(sem_mesh *mesh, sem_pmg *pmg, const double *b_host, double *x_host,
                          const sem_solve_desc *desc, sem_solve_info *info, void *stream);

/* Projection onto previous solutions (Sec. 3, "Projection is key"): the
 * handle keeps an A-orthonormal basis P = [p_1 .. p_L] of earlier solutions
 * and A p_i (FP64 E-layout, 2 Lmax + 3 vectors of n_local owned by the
 * handle, allocated at creation).  sem_solve_projected computes the best fit
 * xbar = P P^T b (one multi-dot), solves A dx = b - A xbar with the solver of
 * desc to the tolerance tol ||b|| (relative to the original b), returns
 * x = xbar + dx (x is output only), and adds dx to the basis after one
 * classical Gram-Schmidt pass in the A-inner product (||p||_A from the same
 * reduction: dx^T A dx - sum alpha_i^2).  When L reaches Lmax the basis
 * restarts from the new solution alone.  info->res0 is ||b - A xbar||,
 * info->iters the iterations of the correction solve.  The handle refers to
 * the mesh, which must outlive it.  Lmax: 1..31. */
typedef struct sem_proj sem_proj;
sem_status sem_proj_create(sem_mesh *mesh, int32_t Lmax, void *stream, sem_proj **out);
sem_status sem_proj_destroy(sem_proj *proj);
/* Number of basis vectors now held (HOST output). */
sem_status sem_proj_info(const sem_proj *proj, int32_t *nvec);
sem_status sem_solve_projected(sem_mesh *mesh, sem_pmg *pmg, sem_proj *proj, const double *b,
                               double *x, const sem_solve_desc *desc, sem_solve_info *info,
                               void *stream);

/* ---- Serving: many independent solves with continuous batching ----------
 * The paper has no counterpart (it runs one large solve across partitions);
 * this is a service of the library for streams of small and mid-sized
 * problems.  A server owns `workers` host threads, each with its own CUDA
 * stream.  A worker takes the oldest queued request whose device memory fits
 * in what the budget leaves (the oldest request runs anyway when nothing else
 * does); a request's memory is the measured bytes of its shape's earlier
 * setup, else the largest bytes per local point measured for its order times
 * its points (+5 %), else, before any setup of its order, 200 bytes per local
 * point + 64 MiB, and a new setup's reservation is replaced by its measured
 * bytes after its first solve; takes an idle setup of the same shape from the cache or
 * builds the mesh and pMG hierarchy (orders N, ceil(N/2), 1), solves, copies x
 * back, and records the result; its next request starts as soon as it is done
 * (continuous batching).  Solves of different workers overlap on the GPU.
 * Every solve is deterministic: results do not depend on the worker count. */
typedef struct sem_server sem_server;

typedef struct {
  int32_t workers;        /* host threads / CUDA streams, 1..64 */
  int64_t hbm_budget;     /* device bytes the server's setups may hold (0: 80 %
                             of the free device memory at creation) */
  int32_t cache_per_shape;/* idle setups kept per mesh shape (0: none) */
  int32_t cheb_degree;    /* pMG template (as sem_pmg_desc; coarse: multigrid
                             CG for N = 1 coarsest levels) */
  int32_t smoother_dtype;
  double coarse_tol;
  int32_t coarse_maxit;
} sem_server_desc;

enum { SEM_RHS_HOST = 0, SEM_RHS_MANUFACTURED = 1 };
typedef struct {
  int32_t ex, ey, ez, N, bc;  /* mesh: box with the built-in jittered vertices */
  double jitter;
  uint64_t seed;
  int32_t rhs;          /* SEM_RHS_HOST: b below; SEM_RHS_MANUFACTURED:
                           b = mask gs(B f), f = 3 pi^2 sin(pi x) sin(pi y)
                           sin(pi z) (Dirichlet only), built on the device */
  const double *b;      /* HOST, n_local values, copied at submit */
  double *x;            /* HOST, n_local values written at completion (may be
                           NULL); must stay valid until the request is polled */
  sem_solve_desc solve; /* PCG, FLEXCG or FGMRES (pMG used for the latter two) */
} sem_request;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t setups_built, setups_reused;
  int64_t hbm_in_use;   /* device bytes of running and cached setups (measured
                           once a setup has solved) */
} sem_server_stats;

sem_status sem_server_create(const sem_server_desc *desc, sem_server **out);
/* Waits for every accepted request, then frees everything. */
sem_status sem_server_destroy(sem_server *server);
/* Queue a request; *ticket identifies it.  SEM_EINVAL for malformed requests
 * (checked at submit), SEM_EBUSY if the queue holds 65,536 requests. */
sem_status sem_submit(sem_server *server, const sem_request *req, uint64_t *ticket);
/* SEM_EAGAIN while pending.  When done: fills *out (out->status is the
 * solve's status, out->time_ms the latency from submit to completion),
 * returns SEM_OK and forgets the ticket.  Unknown ticket: SEM_EINVAL. */
sem_status sem_poll(sem_server *server, uint64_t ticket, sem_solve_info *out);
sem_status sem_server_stats_read(const sem_server *server, sem_server_stats *out);

/* Autotuner: runs the n sample requests (x outputs may be NULL) through
 * servers of 1, 2, 4, ... up to max_workers workers and returns the worker
 * count with the highest throughput (*best_rate in solves per second). */
sem_status sem_server_autotune(const sem_server_desc *base, const sem_request *reqs, int32_t n,
                               int32_t max_workers, int32_t *best_workers, double *best_rate);

/* ---- Batched solves: many independent problems in one graph launch -----
 * The paper has no counterpart (it runs one large solve across partitions);
 * this is a service of the library for many small and mid-sized problems,
 * whose kernels, each alone, would leave most of the GPU idle.
 * sem_batch_create builds every problem's mesh, pMG hierarchy (orders N,
 * N/2 when it lies strictly between 1 and N, and 1; coarse solve:
 * multigrid-preconditioned CG in one cooperative kernel of coarse_ctas CTAs),
 * right-hand side and work vectors in one device arena (a few cudaMalloc
 * calls for the whole batch, no allocation per problem), runs one warm-up
 * solve per distinct order, and captures one CUDA graph that holds every
 * problem's whole FlexCG solve from x = 0 as an independent branch: the
 * V-cycles, operators, inner products and stopping tests run on the device
 * (a conditional node per problem for its iterations), concurrently across
 * problems.  sem_batch_solve launches that graph once, copies each x to the
 * request's host x (when not NULL) and returns every problem's
 * sem_solve_info.  Each x equals, bit for bit, sem_solve (FlexCG, zero
 * guess) on a mesh built from the request and a pMG built from
 * sem_batch_pmg_desc(batch, i), whatever the other problems and ax_fill
 * are.  Requests: SEM_SOLVER_FLEXCG only, 2 <= N <= SEM_MAX_ORDER, SEM_RHS_HOST
 * (b copied at creation; mean-free under Neumann) or SEM_RHS_MANUFACTURED;
 * their x pointers must stay valid while the batch solves. */
typedef struct sem_batch sem_batch;
typedef struct {
  int32_t cheb_degree;      /* pMG template (as sem_pmg_desc) */
  int32_t smoother_dtype;
  double coarse_tol;
  int32_t coarse_maxit;
  int32_t coarse_ctas;      /* CTAs of each coarse solve (0: 1) */
  float ax_fill[SEM_MAX_ORDER + 1];
                            /* per level order: work units (x-line segments)
                               of the FP32 operator per resident CTA slot of
                               the GPU; 0 = 2 (the single-problem default);
                               below 1 a problem's operator also takes only
                               that share of the slots.  Moves work between
                               CTAs only: results do not change. */
  int64_t arena_chunk;      /* bytes per device arena chunk (0: 1 GiB) */
} sem_batch_desc;
/* Errors: SEM_EINVAL (descriptions), SEM_ENOMEM, SEM_ECUDA.  Synchronises. */
sem_status sem_batch_create(const sem_batch_desc *desc, const sem_request *reqs, int32_t n,
                            void *stream, sem_batch **out);
/* infos: HOST array of n entries (may be NULL).  Returns SEM_OK when every
 * problem converged, else the first problem's failing status (SEM_ENOTCONV,
 * SEM_ENUMERIC, SEM_ETIMEOUT); infos hold each problem's.  Synchronises. */
sem_status sem_batch_solve(sem_batch *batch, sem_solve_info *infos, void *stream);
/* Device bytes of the arena, nodes of the graph's top level, host time of
 * the setup in ms (any output may be NULL). */
sem_status sem_batch_info(const sem_batch *batch, size_t *dev_bytes, int32_t *graph_nodes,
                          double *setup_ms);
/* The pMG description of problem i (to reproduce its solve with sem_solve). */
sem_status sem_batch_pmg_desc(const sem_batch *batch, int32_t i, sem_pmg_desc *out);
/* Device address of problem i's solution (owned by the batch). */
sem_status sem_batch_x(const sem_batch *batch, int32_t i, const double **x_dev);
sem_status sem_batch_destroy(sem_batch *batch);
/* Autotuner of the batch's work split, by coordinate descent on the whole
 * batch: starting from the batch's current ax_fill, for one fine order at a
 * time every candidate value (for the levels of that order) is captured into
 * the whole batch's graph and timed (median of reps launches, CUDA events),
 * and the value with the fastest whole-batch time is kept (the current one
 * unless a candidate beats it by more than 2 %).  The tuned values are then
 * timed twice more, alternately with the starting ones, and kept only if
 * they are still faster by that margin.  The batch keeps the graph of the
 * chosen values; they are written to chosen[0..SEM_MAX_ORDER] (HOST, 0 = the
 * default) and *best_ms is the median time of one launch.  Synchronises. */
sem_status sem_batch_autotune(sem_batch *batch, const float *candidates, int32_t ncand,
                              int32_t reps, void *stream, float *chosen, double *best_ms);

/* Tracing (Sec. 4 reports timing breakdowns from CUDA events): while enabled,
 * every kernel launch of the library is counted under a class name such as
 * "ax_f64_N7" or "gs_f32_N3"; launches of classes whose name contains
 * `timed_filter`, or one of its '|'-separated parts (NULL or "" = none, "*" =
 * all), are also bracketed by CUDA events on their stream.  sem_trace_read synchronises on the pending events and fills
 * up to max_entries entries (HOST array); *n_entries receives the number of
 * classes.  reset != 0 clears the counters afterwards. */
typedef struct {
  char name[48];
  int64_t launches;  /* launches counted */
  int64_t timed;     /* launches timed with events */
  double total_ms;   /* summed device time of the timed launches */
} sem_trace_entry;
sem_status sem_trace_enable(int32_t enable, const char *timed_filter);
sem_status sem_trace_read(sem_trace_entry *out, int32_t max_entries, int32_t *n_entries,
                          int32_t reset);

/* Message of the last failed call on this thread ("" if none). */
const char *sem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
