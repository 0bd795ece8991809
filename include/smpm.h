/*
 * smpm.h -- C ABI of libsmpm.so: deflated block-Jacobi Schur-complement GMRES
 * for the SMPM (spectral multidomain penalty, GLL collocation) discretisation
 * of the 2-D Poisson-Neumann problem and of the per-Fourier-mode 2-D
 * Helmholtz problems (Joshi, Thomsen & Diamessis, arXiv:1512.01756).
 *
 * Problem (Sec. 1, Eq. poisson; Sec. 5, Eq. fourier_poisson):
 *     lap u - k^2 u = f  on [0,lx] x [0,lz],   n . grad u = g  on the boundary,
 * discretised by Eq. smpm_poisson on an mx x mz element mesh with n = order+1
 * GLL points per direction, and solved through the Schur complement
 * S = I + B A^-1 E of the strip split L = A + E B (Sec. 2.3, Eq. operator_decomp)
 * with right block-Jacobi preconditioning and deflation (Sec. 3, Alg. seq).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Node order (r = n*n*mx*mz values): index = X*fz + Z with X = ex*n + a the
 *   global x-node (element ex, GLL point a) and Z = ez*n + b the global z-node,
 *   fz = n*mz.  smpm_node_coords() returns the coordinates in this order.
 * Neumann data g (nb = 2*fz + 2*n*mx values): [west: fz][east: fz]
 *   [south: n*mx][north: n*mx]; g = n.grad u with n the outward normal; a corner
 *   node sees the g of both sides it lies on.  A NULL g means g = 0.
 * Pointers: f, g and u may be device pointers or host pointers (pageable or
 *   pinned); the library detects which (cudaPointerGetAttributes) and stages
 *   host buffers through device memory it owns, copying inside the call.
 * Streams: all device work of a handle runs on the stream given at setup
 *   (NULL = the legacy default stream).  Calls on one handle must not overlap.
 * Ownership: the caller owns f, g and u.  The handle owns every operator,
 *   Krylov basis and work array; smpm_release() frees them.
 * Errors: every int-returning call returns SMPM_OK (0) or a negative code;
 *   smpm_last_error() gives a message for the calling thread's last failure.
 *   No C++ exception crosses this boundary.
 * Gauge: for k^2 = 0 the solution is returned with zero GLL-quadrature mean
 *   (the Neumann problem fixes u only up to a constant, Sec. 2.4).
 * Environment switches (none changes a result beyond rounding):
 *   SMPM_TRACE_SETUP / SMPM_TRACE_SOLVE / SMPM_TRACE_PHASES print setup
 *   phases, per-cycle residuals and a solve's phase times on stderr (the last
 *   synchronises the stream at every phase); SMPM_OZAKI (bit mask, read at
 *   setup): 1 runs the FP64 Schur and block-Jacobi products on the tensor
 *   cores at FP64 accuracy, 2 the FP32 products of precisions 1 and 2 at FP32
 *   accuracy; SMPM_COARSE_DENSE=1 (setup) takes the dense factorisation of
 *   the coarse matrix instead of the tridiagonal one; SMPM_INNER_FP64_ARNOLDI=1
 *   keeps the inner Arnoldi arithmetic of precision 2 in FP64;
 *   SMPM_NO_GRAPHS disables CUDA-graph replay of the
 *   Arnoldi steps; SMPM_TILE_SHAPE=0|1 forces a GEMM tile shape instead of
 *   the autotuned one; SMPM_REFINE_EXTENDED forces extra-precise refinement;
 *   SMPM_INNER_STEPS sets the inner steps of precision 2; SMPM_MIRROR=0|1
 *   (read at setup) turns the mirror-symmetric half-size products of the
 *   interior strips, block-Jacobi pairs and slot inverses off, or on at every
 *   batch size (by default S and M^-1 use them where they save enough work);
 *   SMPM_PERSISTENT=1 runs the Arnoldi steps of a restart cycle in one
 *   persistent cooperative kernel (grid-wide barriers between the phases)
 *   instead of graph-replayed step groups of separate launches (the
 *   default, measured faster); SMPM_PERSIST_WAIT_NS sets the time limit of
 *   one grid-barrier wait of that kernel (default 2e9 ns).  Test hook (it only
 *   makes the solve fail): SMPM_PERSIST_STALL=1 makes every barrier wait for
 *   one block more than the grid holds, so the first wait runs out of time
 *   and the solve returns SMPM_ETIMEOUT.
 */
#ifndef SMPM_H
#define SMPM_H

#ifdef __cplusplus
extern "C" {
#endif

#define SMPM_OK 0
#define SMPM_EINVAL (-1)      /* bad argument or size                         */
#define SMPM_ENOMEM (-2)      /* device allocation or admission refused        */
#define SMPM_ENOCONV (-3)     /* max_iter reached; u holds the best iterate     */
#define SMPM_EBREAKDOWN (-4)  /* NaN/Inf or Arnoldi breakdown                  */
#define SMPM_ECUDA (-5)       /* a CUDA / cuSOLVER call failed                 */
#define SMPM_EBUSY (-6)       /* smpm_poll: request still running              */
#define SMPM_ETIMEOUT (-7)    /* a device-side wait gave up (the persistent kernel's
                                 grid barrier); the context stays usable       */

typedef struct smpm_solver* smpm_handle;

/* Grid and solver options.  Defaults used when a field is 0: tau_scale -0.1,
 * z_ratio 1, restart 64, max_iter 2000.  tau_scale is signed in the
 * convention of Eq. smpm_poisson; negative values damp inter-element jumps
 * (|tau_scale| below ~0.028 leaves anti-damped jump modes at orders >= 8). */
typedef struct {
    int mx, mz, order;      /* elements in x and z, polynomial order (n = order+1)   */
    double lx, lz;          /* domain [0,lx] x [0,lz]                                */
    double z_ratio;         /* geometric z-stretch h_{e+1} = z_ratio h_e, 1 = uniform */
    double tau_scale;       /* penalty tau = tau_scale*(N(N+1)/h_perp)^2 on every edge */
    int deflation_groups;   /* 0: one deflation vector per interface (Sec. 3.3);
                               1: one per interface and element row                  */
    int restart;            /* GMRES restart length m                                */
    int max_iter;           /* GMRES iteration cap per solve                         */
    int precision;          /* 0: FP64 throughout; 1: mixed -- FP64 flexible GMRES
                               (Schur product, deflation, CGS2 Arnoldi, Givens,
                               true residual, projections, strip solves) with the
                               block-Jacobi preconditioner in FP32 (FP32 blocks,
                               FP32 accumulation); 2: nested mixed -- FP64
                               flexible GMRES on S (true residual, projections,
                               strip solves in FP64) preconditioned by an inner
                               deflated block-Jacobi GMRES whose Schur products
                               and block-Jacobi applies use FP32 blocks with FP32
                               accumulation (its block-Jacobi inverses are
                               factorised in FP32 too; 10 inner steps or 1e-4 relative;
                               SMPM_INNER_STEPS overrides the step count) and whose
                               CGS2 projections and dot products use FP32
                               arithmetic on FP64-stored vectors
                               (SMPM_INNER_FP64_ARNOLDI=1 keeps them FP64)      */
    int krylov;             /* 0: every right-hand side (every Fourier mode's real
                               and imaginary part) keeps its own Krylov space and
                               meets tol itself; 1: the right-hand sides of one
                               solve call form one concatenated vector and one
                               GMRES runs on the block-diagonal operator (Sec. 5,
                               Implementation; Alg. 3d line 7: all wavenumbers
                               in one GMRES): every dot product and norm is summed
                               over them, and the test is ||[r_1 .. r_R]|| <=
                               tol ||[b_1 .. b_R]|| (a column of small norm may
                               end above tol relative to itself).  The serving
                               runtime refuses 1 (SMPM_EINVAL).                */
} smpm_grid;

typedef struct {
    int iters;              /* GMRES iterations (max over the batch)            */
    int restarts;           /* restart cycles beyond the first                  */
    int status;             /* SMPM_OK / SMPM_ENOCONV / SMPM_EBREAKDOWN         */
    double rel_resid_true;  /* max over the batch of ||S x_S - b_S|| / ||b_S||  */
    double setup_ms;        /* operator build time of the handle                */
    double solve_ms;        /* wall time of this call                           */
} smpm_stats;

/* Build the operators for one k^2 (Sec. 2.3, Sec. 3.2-3.3, Sec. 5 Eq.
 * transverse_schur): strip operators A_c(k) = A_c - k^2 I and their inverses per
 * strip class, the Schur blocks G_c = B A_c^-1 E, the block-Jacobi pair blocks
 * and their inverses, the deflation coarse operator, and for k2 = 0 the left
 * null vectors u_L, u_S (Claim 1).  stream: a cudaStream_t or NULL.
 * Returns SMPM_EINVAL for mx < 2, mz < 1, order < 1, order > 32, k2 < 0. */
int smpm_setup(const smpm_grid* grid, double k2, void* stream, smpm_handle* out);

/* Solve L u = f + tau g (Alg. seq) for one right-hand side to a relative
 * Schur residual ||S x_S - b_S|| / ||b_S|| <= tol (the paper's check, Sec. 4).
 * f, u: r doubles; g: nb doubles or NULL.  st may be NULL. */
int smpm_solve(smpm_handle h, const double* f, const double* g, double tol,
               double* u, smpm_stats* st);

/* Solve nrhs independent right-hand sides with the same operator in one
 * batched pass: f and u hold nrhs consecutive r-vectors, g nrhs consecutive
 * nb-vectors (or NULL).  Each right-hand side keeps its own Krylov space and
 * meets tol itself. */
int smpm_solve_batch(smpm_handle h, int nrhs, const double* f, const double* g,
                     double tol, double* u, smpm_stats* st);

/* smpm_solve_batch from an initial guess u0 (nrhs consecutive r-vectors, host
 * or device; NULL = zero): the first refinement cycle starts from
 * x_S0 = B u0, the interface unknowns of the guess (the exact solution has
 * x_S = B u, Sec. 2.3), so a guess close to the solution (the previous time
 * step's field) leaves only its error for GMRES.  The convergence test is the
 * same (||S x_S - b_S|| <= tol ||b_S||).  The guess is ignored on the
 * dense-inverse fallback path. */
int smpm_solve_guess(smpm_handle h, int nrhs, const double* f, const double* g, const double* u0,
                     double tol, double* u, smpm_stats* st);

/* One handle holding the operators of several k^2 values (the Fourier modes
 * of the 3-D problem, Sec. 5, Alg. 3d): nop >= 1 values k2[0..nop-1], at most
 * one of them zero.  Each operator set is built as by smpm_setup. */
int smpm_setup_multi(const smpm_grid* grid, int nop, const double* k2, void* stream,
                     smpm_handle* out);

/* Batched solve over right-hand sides that use different operator sets of a
 * multi handle: right-hand side i uses operator op_of_rhs[i] (non-decreasing,
 * in [0, nop)).  All of them run in the same kernel launches (the per-mode
 * Schur products, block-Jacobi applies and Arnoldi steps of Alg. 3d batched),
 * each with its own Krylov space and convergence test.  Layouts as in
 * smpm_solve_batch. */
int smpm_solve_multi(smpm_handle h, int nrhs, const int* op_of_rhs, const double* f,
                     const double* g, double tol, double* u, smpm_stats* st);

/* Apply one operator of the method (operator set 0) to nrhs vectors, for
 * checking the individual kernels.  kind 0: y = S x, the Schur product
 * (Sec. 2.3, Eq. operator_decomp; assembled form of Sec. 3.1); 1: y = M^-1 x,
 * block-Jacobi (Sec. 3.2); 2: y = P x = x - S Z K Z^T x, the deflation
 * projection with the regularised coarse division K (Sec. 3.3); 3: y = B A^-1 b
 * (the Schur right-hand side map, Alg. seq step 2; in: r-vectors, out:
 * k-vectors); 4: y = A^-1 b (strip solves, r -> r).  k-vectors use the
 * interface order (2 j + s) fz + Z: interface j = 0..mx-2, side s = 0 the
 * east face of strip j, s = 1 the west face of strip j+1.  Pointers host or
 * device; in and out hold nrhs consecutive vectors. */
int smpm_apply(smpm_handle h, int kind, int nrhs, const double* in, double* out);

/* 3-D y-periodic problem (Sec. 5, Eqs. poisson3d / fourier_poisson, Alg. 3d)
 * in Fourier space: u(x,y,z) = sum_j u_j(x,z) e^{i k_j y}, k_j = 2 pi j / ly,
 * j = 0 .. my/2 (my even).  Each mode is the 2-D Helmholtz problem
 * (L - k_j^2) u_j = f_j with its own Schur operator S(k_j) (Eq.
 * transverse_schur), block-Jacobi and deflation; mode 0 is the singular
 * Poisson-Neumann problem with the null-space projections.  setup builds the
 * my/2+1 operator sets; solve runs every mode's real and imaginary parts as
 * separate right-hand sides in the same kernel launches, each with its own
 * Krylov space and convergence test.
 * fhat, uhat: [my/2+1][2 (re, im)][r] doubles; ghat: [my/2+1][2][nb] or NULL.
 * The y-transform itself (a real DFT of length my per node) is the caller's. */
int smpm_setup_3d(const smpm_grid* grid, int my, double ly, void* stream, smpm_handle* out);
int smpm_solve_3d(smpm_handle h, const double* fhat, const double* ghat, double tol,
                  double* uhat, smpm_stats* st);

/* The same 3-D problem in physical space (Alg. 3d with the y-transforms on the
 * GPU): f3, u3: [my][r] doubles, plane t holding the samples at
 * y_t = t ly / my in node order; g3: [my][nb] Neumann data per plane, or NULL.
 * The real DFT along y (u_j = (1/my) sum_t u(y_t) e^{-2 pi i j t/my}), the
 * batched mode solve of smpm_solve_3d and the inverse DFT run on the handle's
 * stream; pointers host or device.  Only for handles from smpm_setup_3d
 * (SMPM_EINVAL otherwise).  st->solve_ms covers the whole call. */
int smpm_solve_3d_physical(smpm_handle h, const double* f3, const double* g3, double tol,
                           double* u3, smpm_stats* st);

/* Number of nodes r, Neumann values nb and Schur unknowns k of a handle. */
int smpm_sizes(smpm_handle h, long long* r, long long* nb, long long* k);

/* Node coordinates in node order (x and z: r doubles each, host memory).
 * smpm_grid_coords gives the same for a grid without building a handle
 * (host work only; SMPM_EINVAL for a grid smpm_setup would reject). */
int smpm_node_coords(smpm_handle h, double* x, double* z);
int smpm_grid_coords(const smpm_grid* grid, double* x, double* z);

/* Per right-hand side relative Schur residual ||S x_S - b_S|| / ||b_S|| of the
 * handle's last solve (first n of them, host memory). */
int smpm_last_residuals(smpm_handle h, int n, double* out);

/* Left null vectors of the k^2 = 0 operator set (Claim 1): u_L (r doubles,
 * node order, unit norm, L^T u_L = 0) and u_S = E^T u_L / |E^T u_L| (k doubles,
 * interface order as in smpm_apply).  Host or device pointers.  SMPM_EINVAL if
 * the handle has no k^2 = 0 operator set. */
int smpm_null_vectors(smpm_handle h, double* uL, double* uS);

/* Move a handle's device work to another stream (a cudaStream_t or NULL);
 * waits for the work queued on the old stream first.  Lets a handle built on
 * one thread's stream be reused from another's. */
int smpm_set_stream(smpm_handle h, void* stream);

/* Device bytes held by the handle (operators + workspace). */
long long smpm_device_bytes(smpm_handle h);

void smpm_release(smpm_handle h);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (an
 * independent-chain DFMA loop over 8 blocks per SM); the FP64 roofline
 * denominator of the dense applies.  stream: cudaStream_t or NULL. */
int smpm_probe_fp64(void* stream, double* tflops);

/* Profiling of the dense class-GEMM launches (the Schur products, block-Jacobi
 * applies and strip solves): when enabled, every such launch is bracketed by
 * CUDA events on the handle's stream and its algorithmic FLOPs
 * (2 x stored rows x K x active columns of a full product, 4 x rows x h x
 * active columns of a mirror-form one) are counted on the device.
 * smpm_profile_read returns the totals since the last reset (h = NULL: the
 * totals of every handle of the process).  Profiling turns graph replay off
 * while it is enabled. */
int smpm_profile(smpm_handle h, int enable);
int smpm_profile_read(smpm_handle h, long long* launches, double* flops, double* ms, int reset);
/* The same totals split by the kind of launch (precision 0: FP64 products
 * on the CUDA cores, 1: FP32 products of the mixed forms, 2: FP64-accurate
 * tensor-core products, SMPM_OZAKI=1, with their algorithmic FLOPs, 3: the
 * same launches' executed BF16 tensor-core FLOPs, their time under 2).
 * h = NULL reads the totals of every handle of the process (harvested at the
 * end of each solve), and smpm_profile(NULL, enable) makes every handle
 * created afterwards profile (the serving workers' handles included).
 * SMPM_EINVAL for another kind. */
int smpm_profile_split(smpm_handle h, int precision, long long* launches, double* flops, double* ms, int reset);

/* Number of CUDA kernels this library has launched in the process. */
long long smpm_kernel_launches(void);

/* Allocation-free deflation projection (no counterpart in the paper; an
 * interface for callers that cannot allocate device memory when they call:
 * real-time loops, such as a time stepper projecting every step, that must
 * not meet the allocator's latency or the device-wide synchronisation that
 * cudaMalloc / cudaFree can cause, and host applications that give the
 * library a fixed device-memory budget up front and own every allocation).
 * Computes y = P x = x - S Z K Z^T x for operator set 0 of h -- the same
 * result as smpm_apply(h, 2, ...) -- without calling cudaMalloc, cudaFree or
 * any allocating library routine.
 *   x, y: device pointers to nrhs consecutive k-vectors (interface order as in
 *         smpm_apply); y may equal x (in place); host pointers are rejected
 *         with SMPM_EINVAL.
 *   Scratch: a fixed device array of SMPM_NOALLOC_MAX_DOUBLES doubles inside
 *         the library, held by every GPU that loads it until the process
 *         exits; a call needs 2 * nrhs * d of them (d = (mx - 1) per-interface
 *         deflation groups, or (mx - 1) mz) and is rejected with SMPM_EINVAL
 *         above that.  All calls share the array and it keeps the last call's
 *         contents (each call writes every entry it reads first); calls whose
 *         kernels overlap on the GPU race on it, so order them on one stream.
 *   The first call on a device looks up the array's device address
 *         (cudaGetSymbolAddress) and keeps it for the process, which assumes
 *         the device's primary context is not reset (cudaDeviceReset) while
 *         the library is in use; make that first call before any stream
 *         capture.  Work is queued on the handle's stream; the call returns
 *         without synchronising. */
#define SMPM_NOALLOC_MAX_DOUBLES 65536
int smpm_apply_deflation_noalloc(smpm_handle h, int nrhs, const double* x, double* y);

/* Serving runtime (continuous batching; no counterpart in the paper, which
 * solves one problem at a time).  A server owns nworkers host threads, each
 * with its own CUDA stream on the device current at create time.
 * smpm_submit() queues one solve of L u - k2 u = f + tau g on the given grid
 * (Sec. 2.3, Alg. seq; the Helmholtz form of Sec. 5) and returns a ticket at
 * once.  A free worker takes the oldest pending request together with up to
 * max_batch - 1 other pending requests of the same grid options and tol (any
 * k2), builds one multi-operator handle for their distinct k2 values
 * (smpm_setup_multi) and solves them in one batched call (smpm_solve_multi):
 * each request keeps its own Krylov space and convergence test, so its result
 * is the one a lone smpm_setup + smpm_solve gives, to the solver tolerance.
 * Requests that arrive while batches run are taken by the next free worker and
 * run concurrently with them on its stream.  Admission: a batch starts only if
 * its estimated device footprint (operators of each k2, Krylov bases and work
 * vectors per request) fits device_budget_bytes beside the batches in flight
 * (<= 0: 80 % of the free device memory at create time); a batch that fits
 * nowhere runs alone, and a request whose own footprint exceeds the budget is
 * refused: smpm_submit still returns SMPM_OK and a ticket, and smpm_poll
 * reports SMPM_ENOMEM for it.  grid->krylov must be 0 (SMPM_EINVAL otherwise):
 * requests batched together keep their own Krylov spaces.
 *   f, g, u: host or device pointers of r, nb and r doubles, owned by the
 *   caller, which must keep them valid and unchanged until smpm_poll() has
 *   returned something other than SMPM_EBUSY for the ticket.  g may be NULL.
 *   smpm_poll(): SMPM_EBUSY while the request is pending or running; else the
 *   solve's status, with st (may be NULL) filled: iters and rel_resid_true of
 *   the request, setup_ms of its batch, solve_ms = completion - submission
 *   (wall ms, setup included), restarts = the number of requests in its batch.
 *   A ticket is forgotten once it has been polled to completion.
 *   smpm_server_destroy(): finishes every queued request, joins the workers
 *   and frees the server. */
typedef struct smpm_server* smpm_server_t;
int smpm_server_create(int nworkers, long long device_budget_bytes, int max_batch, smpm_server_t* out);
int smpm_submit(smpm_server_t srv, const smpm_grid* grid, double k2, const double* f, const double* g,
                double tol, double* u, unsigned long long* ticket);
int smpm_poll(smpm_server_t srv, unsigned long long ticket, smpm_stats* st);
int smpm_server_destroy(smpm_server_t srv);

/* The estimated device footprint the admission above charges for a batch of
 * nrhs requests with nop distinct k2 values on grid (bytes, written to
 * *bytes): a caller sizes device_budget_bytes with it.  SMPM_EINVAL for a
 * null argument, nop < 1 or nrhs < 1.  Host arithmetic only (no GPU call). */
int smpm_request_footprint(const smpm_grid* grid, int nop, int nrhs, long long* bytes);

/* Residual history of right-hand side `rhs` of the handle's last solve
 * (tracing; Sec. 4 reports convergence as the relative residual per
 * iteration).  kind 0: after every Arnoldi step of every restart cycle, the
 * GMRES residual estimate |g_{j+1}| / ||b_S|| from the Givens rotations (of
 * the deflated, preconditioned cycle system; written on the device by the
 * normalisation kernel, outer iteration of the nested form); kind 1: at every
 * restart-cycle start while the right-hand side was running, the recomputed
 * true residual ||S x_S - b_S|| / ||b_S||.  Writes min(n, available) values
 * to out (host memory) and the number available to *count; n = 0 queries the
 * count (out may then be NULL).  SMPM_EINVAL for a null handle or count, rhs
 * outside the last solve, a bad kind, n < 0 or out NULL with n > 0.  Valid
 * until the next solve on the handle. */
int smpm_residual_history(smpm_handle h, int rhs, int kind, int n, double* out, int* count);

/* Message of the calling thread's last failure ("" if none). */
const char* smpm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SMPM_H */
