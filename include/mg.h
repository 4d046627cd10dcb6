/*
 * mg.h -- C ABI of the GB300 multigrid-preconditioned CG library.
 *
 * The library solves A x = b (Eq. 1) where A is the 7-point discretisation of
 * the heat-conduction operator -div(k grad phi) = f (Eq. 2) on a vertex-centred
 * structured grid of the unit cube with zero Dirichlet boundary values.  The
 * preconditioner is one geometric-multigrid V-cycle (Algorithm 1 applied
 * recursively; per-level components of Sec. 2.1.1) with re-discretised coarse
 * operators (Sec. 1, Sec. 4.3), a Jacobi-preconditioned Chebyshev smoother
 * (Sec. 4.3), full-weighting restriction, trilinear prolongation, and an exact
 * dense Cholesky solve of the coarsest operator (Sec. 1, Sec. 3.3.1).  Coarse
 * levels too small to fill the GPU run on progressively fewer thread blocks and
 * finally inside one persistent thread block: the single-GPU analogue of
 * agglomerating a coarse problem onto fewer ranks (Sec. 3, Sec. 3.1).  The
 * outer Krylov method is CG (Sec. 2.1), stopped when the residual 2-norm falls
 * below rtol times that of b (Sec. 4.2, Sec. 4.3).
 *
 * Conventions shared by every entry point:
 *  - Grids are given by their vertex counts Nx, Ny, Nz, boundary included.
 *    Each N-1 must be divisible by 2^(levels-1); the coarsest level keeps at
 *    least 3 interior points per axis and at most MG_MAX_COARSE unknowns.
 *  - Nodal arrays (f, x, g, lambda, phi, ...) are dense C-order [z][y][x]
 *    float64 arrays of Nz*Ny*Nx entries, x fastest.  Boundary entries of inputs
 *    are ignored; boundary entries of outputs are written as 0.
 *  - Cell arrays (k, gradients) are dense [z][y][x] float64 arrays of
 *    (Nz-1)*(Ny-1)*(Nx-1) entries, cell (ci,cj,ck) having lower corner vertex
 *    (ci,cj,ck).
 *  - All array pointers are DEVICE pointers owned by the caller unless stated
 *    otherwise; the library never frees them.  The handle owns its internal
 *    level buffers and releases them in mg_free.
 *  - Work is enqueued on the CUDA stream given to mg_setup (or mg_set_stream).
 *    Entry points that return results to the host (mg_solve, the statistics)
 *    synchronise that stream before returning; the step entry points do not.
 *  - Every call returns an mg_status; no C++ exception crosses the ABI.  The
 *    message of the last failure is available from mg_last_error.
 */
#ifndef MG_H
#define MG_H

#ifdef __cplusplus
extern "C" {
#endif

#define MG_MAX_LEVELS 16
#define MG_MAX_COARSE 1024
#define MG_MAX_SLABS 64

typedef struct mg_handle mg_handle; /* opaque; owned by the library */

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = 1,             /* invalid argument (dims, levels, pointers, params) */
  MG_ERR_ALLOC = 2,           /* device allocation failed */
  MG_ERR_CUDA = 3,            /* a CUDA runtime call or kernel failed */
  MG_ERR_NONFINITE = 4,       /* NaN/Inf in k, f or during the iteration */
  MG_ERR_NOT_CONVERGED = 5,   /* maxit reached; x holds the last iterate */
  MG_ERR_BREAKDOWN = 6,       /* CG breakdown: p.Ap <= 0 */
  MG_ERR_DEVICE_TIMEOUT = 7,  /* a bounded on-device wait gave up */
  MG_ERR_NOT_SPD = 8          /* coarsest operator not positive definite */
} mg_status;

typedef enum {
  MG_FP64 = 0,        /* everything in float64 */
  MG_MIXED_FP32 = 1,  /* V-cycle in float32 (vectors and coefficients) inside float64 CG */
  MG_MIXED_BF16K = 2  /* V-cycle in float32 with bfloat16 edge coefficients inside float64 CG */
} mg_precision;
/* In every form CG's rho is b.z, with z the V-cycle's output and b the finest right-hand side it
 * read: the float64 residual r itself (MG_FP64), or its float32 rounding (mixed forms), which makes
 * rho = b^T M b for the preconditioner M the float32 V-cycle applies.  It is summed in float64
 * (in the mixed forms' default kernel each thread first sums its terms as a compensated float32
 * dot product). */

typedef enum {
  MG_SMOOTHER_CHEBYSHEV = 0,  /* Chebyshev(cheby_degree) preconditioned with Jacobi (Sec. 4.3) */
  MG_SMOOTHER_RICHARDSON = 1  /* Richardson preconditioned with Jacobi, x += omega D^-1 (b - A x)
                                 (Sec. 2.1.1; Sec. 5 runs eight iterations per level) */
} mg_smoother;

typedef enum {
  MG_COARSE_REDISCRETISED = 0, /* coarse operators re-discretised from averaged cell k (Sec. 1, Sec. 4.3) */
  MG_COARSE_GALERKIN = 1       /* Galerkin A_{l+1} = R A_l P, 27-point stencils (Sec. 4.3, Sec. 5); each
                                  Galerkin level's Chebyshev interval is [eig_lo_frac G, G] with G the
                                  Gershgorin bound of its D^-1 A */
} mg_coarse_op;

typedef enum {
  MG_KRYLOV_CG = 0,     /* preconditioned CG (Sec. 2.1) */
  MG_KRYLOV_FGMRES = 1  /* flexible GMRES(gmres_restart), right-preconditioned by the V-cycle; classical
                           Gram-Schmidt; stops on the rotated residual norm (Sec. 5) */
} mg_krylov;

typedef struct {
  int levels;          /* number of levels; 0 = coarsen until an axis has 3 interior points */
  int nu_pre, nu_post; /* smoother sweeps before / after the coarse correction (default 1, 1) */
  int cheby_degree;    /* Chebyshev iterations per sweep, 1..32 (default 2: "V(2,2), Chebyshev(2)") */
  double eig_lo_frac;  /* interval [eig_lo_frac*eig_hi, eig_hi] for D^-1 A (default 0.1) */
  double eig_hi;       /* upper end; 2.0 bounds the spectrum of D^-1 A (Gershgorin) */
  int coarse_k_rule;   /* coarse cell k from its 8 children: 0 arithmetic (default), 1 geometric, 2 harmonic mean */
  int face_rule;       /* edge k from the 4 cells sharing it: 0 harmonic mean (default), 1 arithmetic mean */
  int k_is_log;        /* 1: k_cells holds ln k instead of k */
  mg_precision precision;
  int maxit;           /* CG iteration limit (default 1000) */
  int nonzero_guess;   /* 1: mg_solve starts from the x passed in */
  int flexible;        /* CG beta: 0 Fletcher-Reeves, 1 Polak-Ribiere (flexible); -1 (default) = 0 */
  int telescope_max_n; /* levels with at most this many unknowns run inside the bottom kernel, one thread block
                          or one thread-block cluster (bottom_blocks) (default 4096) */
  int use_graph;       /* 1: replay the V-cycle from a captured CUDA graph (default 1) */
  int stencil_kernel;  /* smoother/residual kernels on the levels above the bottom kernel:
                          0 (default) z-marching, 64x4 tiles of two consecutive points per
                            thread: vector loads, x neighbours by warp shuffles, z neighbours
                            in registers, L2 prefetch two planes ahead (the fastest measured
                            on GB300),
                          1 TMA-staged tiles (cp.async.bulk.tensor into an mbarrier-tracked ring of
                            shared-memory stages; every wait bounded),
                          2 z-marching with one point per thread and neighbours read through L1 (the
                            driver the float64 CG operator and the 27-point passes always use) */
  int use_pdl;         /* 1: launch solve kernels as programmatic dependent launches (default 1) */
  int smoother;        /* mg_smoother (default MG_SMOOTHER_CHEBYSHEV).  With Richardson, nu_pre and
                          nu_post count iterations and cheby_degree, eig_lo_frac, eig_hi are unused */
  double richardson_omega; /* Richardson damping, > 0.  The paper gives none; the default 6/7 is
                              the weight that minimises Jacobi's smoothing factor for the 7-point
                              operator (1.0 leaves the highest modes undamped) */
  int coarse_op;       /* mg_coarse_op (default MG_COARSE_REDISCRETISED) */
  int krylov;          /* mg_krylov (default MG_KRYLOV_CG) */
  int gmres_restart;   /* FGMRES restart length m, 1..256 (default 30); the basis takes (m+1) float64
                          and m V-cycle-precision vectors of the finest level, allocated on first use */
  int eig_mode;        /* Chebyshev interval of every level: 0 (default) [eig_lo_frac b, b] with b = eig_hi
                          (the Gershgorin bound on Galerkin levels); 1 [eig_lo_frac L, eig_safety L] with L
                          a 10-step CG-Lanczos estimate of the largest eigenvalue of D^-1 A on the level,
                          from a seeded random right-hand side (computed at setup) */
  double eig_safety;   /* upper factor of eig_mode 1 (default 1.1) */
  int coarse_solve;    /* coarsest solve: 0 (default) dense Cholesky; 1 GMRES preconditioned with
                          Jacobi, stopped at coarse_rtol (the inexact, truncated coarse solve of Sec. 5;
                          the V-cycle is then no longer a fixed linear operator: use MG_KRYLOV_FGMRES).
                          1 needs a coarsest level of at most 32 unknowns */
  double coarse_rtol;  /* relative residual of the inexact coarse solve (default 1e-4) */
  int coarse_maxit;    /* its iteration limit, 1..32 (default 30) */
  int bottom_blocks;   /* blocks of the bottom kernel: 0 (default) one block, or, in the float64 form and
                          for Galerkin (27-point) bottom levels, one block per 1024 points of its finest
                          level up to a cluster of 8; 1 one block; 2, 4 or 8 one thread-block cluster that
                          splits every pass.  The result is bitwise the same for every choice */
  int test_inject;     /* TEST ONLY: a data perturbation made by the host at setup so that the error paths
                          can be exercised without any GPU fault.  0 (default) none; 1 the float64 finest
                          diagonal used by the outer Krylov operator is negated, so p.Ap < 0 and mg_solve
                          returns MG_ERR_BREAKDOWN in its first iteration; 2 the diagonal of the dense
                          coarsest operator is negated before its Cholesky factorisation, so mg_setup returns
                          MG_ERR_NOT_SPD; 3 the bounded waits of the TMA-staged kernels (stencil_kernel 1)
                          give up without polling, so every block sets the timeout flag, drains the copies
                          it issued (with the full poll limit) and returns, and mg_solve returns
                          MG_ERR_DEVICE_TIMEOUT */
  int slabs;           /* z-slab domain decomposition of the solve (the structured-grid decomposition of
                          Sec. 2.2 with the coarse levels agglomerated onto one hierarchy, Sec. 3.1), 1..MG_MAX_SLABS.
                          1 (default): none.  S > 1: every level above the agglomeration level is split into S
                          runs of consecutive z planes (see mg_slab_plan), each slab holding its planes plus one
                          halo plane per neighbour; every stencil and transfer pass first exchanges its
                          operand's boundary planes with the neighbouring slabs, every dot product is summed per
                          slab and then over the slabs in slab order, and the agglomeration level's right-hand
                          side is gathered into the whole-grid hierarchy, whose V-cycle (bottom kernel) runs
                          from there and whose correction is scattered back.  All slabs run on the handle's
                          device and stream, one after another, each copy standing for a transfer between
                          ranks.  Needs krylov = CG, stencil_kernel 0 or 2, nonzero_guess = 0.  Only mg_solve,
                          mg_solve_host and mg_solve_adjoint use the slabs; the step entry points work on the
                          whole grid */
  int slab_level;      /* agglomeration level of the slabs: 0 (default) the bottom kernel's first level;
                          otherwise that level, at most the bottom kernel's first level, at least 1 */
  int slab_rank;       /* -1 (default): this process holds all slabs.  0..slabs-1: this process holds only
                          slab slab_rank (one process per rank of a distributed run) and exchanges halo
                          planes, dot-product sums and the agglomeration level with the other ranks through
                          the transport given to mg_set_transport; every rank gathers the agglomeration level
                          and runs the whole-grid V-cycle from there itself.  mg_solve then reads all of f and
                          writes only this slab's planes of x (the first and last rank also the boundary
                          planes); statistics are those of the whole solve on every rank */
} mg_params;

typedef struct {
  int iters;             /* CG iterations performed */
  double rel_resid;      /* recurrence residual ||r||/||b|| at exit */
  double true_rel_resid; /* ||b - A x||/||b|| recomputed in float64 at exit */
  double bnorm;          /* ||b||_2 over interior nodes */
  double setup_s;        /* wall time of mg_setup */
  double solve_s;        /* wall time of the last solve */
  long long kernel_launches; /* kernels launched by the last solve (graph replays count their kernels) */
} mg_stats;

/* Fill p with the defaults listed above.  p must be non-NULL. */
mg_status mg_params_default(mg_params* p);

/* Build the level hierarchy for the conductivity field k_cells (one value per
 * finest cell, > 0 and finite; ln k if p->k_is_log).  k_cells is a device
 * pointer if k_on_device, else a host pointer; it is copied, not retained.
 * stream is a cudaStream_t (NULL = default stream).  On success *h owns all
 * device buffers of the hierarchy.  Setup follows Eq. 2 with the face rule of
 * p->face_rule on every level and the coarse rule of p->coarse_k_rule between
 * levels, and factors the coarsest operator with a dense Cholesky. */
mg_status mg_setup(mg_handle** h, int Nx, int Ny, int Nz, const double* k_cells, int k_on_device,
                   const mg_params* p, void* stream);

/* The z-slab partition of mg_params.slabs for a grid (host arithmetic only;
 * needs no device).  On return *agglomerate_level = la and bounds (at least
 * (la+1)*(slabs+1) entries, cap given) holds, for every level l = 0..la and
 * slab s, the slab's first interior z plane (0-based) at bounds[l*(slabs+1)+s],
 * and the level's plane count at bounds[l*(slabs+1)+slabs].  On level la the
 * planes are split as evenly as possible; on finer levels each slab owns the
 * planes 2^(la-l) times its coarse ones (the last slab also the level's final
 * plane), so restriction needs one halo plane above a slab and prolongation
 * one below.  MG_ERR_ARG when the grid, the parameters or cap do not allow it. */
mg_status mg_slab_plan(int Nx, int Ny, int Nz, const mg_params* p, int* bounds, int cap, int* agglomerate_level);

/* Transport between the ranks of a z-slab solve (mg_params.slab_rank >= 0).
 * The caller allocates the device buffers (sizes from
 * mg_slab_transport_sizes) and implements three collective operations over
 * the ranks 0..slabs-1; each is called by every rank in the same order,
 * with the library's stream, and must complete the transfer before the
 * stream's next work (enqueue it on that stream, or finish it before
 * returning).  Every call returns 0 on success.
 *  exchange(ctx, nbytes, has_lo, has_hi, stream): the first nbytes of
 *    send_lo go to rank-1 (into its recv_hi) and of send_hi to rank+1 (into
 *    its recv_lo); recv_lo receives from rank-1 and recv_hi from rank+1.
 *    has_lo / has_hi say whether those neighbours exist.
 *  allreduce(ctx, n, stream): reduce_buf[0..n) becomes its sum over the ranks.
 *  allgather(ctx, block_bytes, stream): gather_recv[r*block_bytes ..) becomes
 *    rank r's gather_send[0 .. block_bytes) for every r. */
typedef struct {
  void* ctx;
  int (*exchange)(void* ctx, long long nbytes, int has_lo, int has_hi, void* stream);
  int (*allreduce)(void* ctx, int n, void* stream);
  int (*allgather)(void* ctx, long long block_bytes, void* stream);
  void *send_lo, *send_hi, *recv_lo, *recv_hi; /* device, plane_bytes each */
  double* reduce_buf;                           /* device, 2 doubles */
  void *gather_send, *gather_recv;              /* device, block_bytes and slabs * block_bytes */
} mg_transport;

/* Buffer sizes of a rank's transport: the largest halo plane and the
 * agglomeration level's largest block of planes, in bytes. */
mg_status mg_slab_transport_sizes(const mg_handle* h, long long* plane_bytes, long long* block_bytes);
/* Set (copy) the transport of a handle built with slab_rank >= 0. */
mg_status mg_set_transport(mg_handle* h, const mg_transport* t);

/* Change the stream subsequent calls enqueue on. */
mg_status mg_set_stream(mg_handle* h, void* stream);

/* Solve A x = f by V-cycle-preconditioned CG until ||r|| <= rtol ||f||.
 * f, x: device nodal arrays.  x is read as the initial guess only when the
 * handle was built with nonzero_guess.  On MG_ERR_NOT_CONVERGED x holds the
 * last iterate.  st may be NULL. */
mg_status mg_solve(mg_handle* h, const double* f, double* x, double rtol, mg_stats* st);

/* Adjoint solve A lambda = g (A is symmetric, so this is mg_solve on g), then,
 * when grad_logk is non-NULL, the gradient of the loss whose derivative with
 * respect to phi is g, taken with respect to the natural log of each finest
 * cell's k:  dL/dln k_c = sum over the 12 edges e=(p,q) of cell c of
 * -h_a^-2 (lambda_p - lambda_q)(phi_p - phi_q) dk_e/dln k_c.  phi is the
 * forward solution (device nodal array, required when grad_logk is non-NULL).
 * dL/df equals lambda.  grad_logk is a device cell array. */
mg_status mg_solve_adjoint(mg_handle* h, const double* g, double* lambda, double rtol,
                           const double* phi, double* grad_logk, mg_stats* st);

/* mg_solve with HOST buffers: f_host and x_host are host nodal arrays (pinned
 * memory gives full-bandwidth copies; pageable memory works, more slowly).
 * The call copies f to the device, solves (x_host is read as the initial
 * guess when the handle was built with nonzero_guess), copies x back and
 * synchronises the stream, all on the handle's stream.  The first call
 * allocates two device nodal arrays of the finest grid, kept by the handle
 * until mg_free.  Errors as mg_solve; on MG_ERR_NOT_CONVERGED x_host holds the
 * last iterate. */
mg_status mg_solve_host(mg_handle* h, const double* f_host, double* x_host, double rtol, mg_stats* st);

/* Release every buffer the handle owns.  h may be NULL. */
mg_status mg_free(mg_handle* h);

/* Message of the last failure on this handle (or of the last failed
 * mg_setup when h is NULL).  Valid until the next call on the handle. */
const char* mg_last_error(const mg_handle* h);

/* ---- introspection ------------------------------------------------------ */
int mg_num_levels(const mg_handle* h);
/* Vertex counts of level l (0 = finest) into N3 = {Nx, Ny, Nz}. */
mg_status mg_level_dims(const mg_handle* h, int l, int* N3);
/* Chebyshev interval [*alpha, *beta] of D^-1 A used by the smoother on level l. */
mg_status mg_level_interval(const mg_handle* h, int l, double* alpha, double* beta);
/* Copy up to cap entries of the last solve's ||r_k||/||b|| history to the
 * host array hist; returns the number available. */
int mg_history(const mg_handle* h, double* hist, int cap);

/* ---- step entry points (one row of the solve each; device nodal arrays of
 * the level's size; computed in the hierarchy's V-cycle precision, inputs
 * rounded to it and outputs widened to float64) -------------------------- */

/* y = A_l x (Eq. 2 re-discretised on level l).  l = -1 selects the float64
 * finest operator used by the outer CG whatever the precision. */
mg_status mg_apply(mg_handle* h, int l, const double* x, double* y);
/* One smoother sweep on level l: cheby_degree Chebyshev iterations for
 * D^-1 A on [eig_lo_frac*eig_hi, eig_hi] (Sec. 4.3).  x is the initial guess
 * unless zero_guess, and is overwritten with the result. */
mg_status mg_smooth(mg_handle* h, int l, const double* b, double* x, int zero_guess);
/* bc = R (b - A_l x): residual then full-weighting restriction R = P^T/8
 * to level l+1 (Algorithm 1, restriction step). */
mg_status mg_residual_restrict(mg_handle* h, int l, const double* b, const double* x, double* bc);
/* x += P ec: trilinear prolongation from level l+1 to level l (Algorithm 1,
 * prolongation step). */
mg_status mg_prolong_add(mg_handle* h, int l, const double* ec, double* x);
/* x = A_L^-1 b on the coarsest level by the dense Cholesky factor. */
mg_status mg_coarse_solve(mg_handle* h, const double* b, double* x);
/* z = M^-1 r: one V-cycle with zero initial guess from the finest level. */
mg_status mg_vcycle(mg_handle* h, const double* r, double* z);
/* Cell gradient dL/dln k from phi and lambda (see mg_solve_adjoint). */
mg_status mg_gradient(mg_handle* h, const double* phi, const double* lambda, double* grad_logk);
/* ||f - A x||_2 on the float64 finest operator, written to *out (host). */
mg_status mg_residual_norm(mg_handle* h, const double* f, const double* x, double* out);

/* ---- residual norm without any device allocation --------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory at the time they check a solution:
 * code running where another memory manager owns the whole device (so a raw
 * cudaMalloc would fail or fragment its pool), or code that must keep a fixed
 * memory footprint.  It computes ||f - A x||_2 over interior nodes with the
 * handle's float64 finest operator, like mg_residual_norm, but reads f and x
 * in their dense nodal layout directly (no copy into the handle's buffers),
 * keeps its per-plane partial sums in a statically sized device array that
 * the library holds for the life of the process, and writes the result to
 * the DEVICE pointer out (one double) without synchronising.
 *  - f, x: device nodal arrays of the handle's finest grid (boundary entries
 *    ignored).  out: device pointer to one double.  All owned by the caller.
 *  - Allocates nothing: no cudaMalloc/cudaFree, no allocating library call.
 *  - Limit: Nz - 2 (interior planes) <= MG_NOALLOC_MAX_PLANES; larger grids
 *    are rejected with MG_ERR_ARG.
 *  - The first call on each device looks up the address of the static array
 *    with that device current; make that first call before any stream
 *    capture.
 *  - Every call shares the one static array (per device): calls that overlap
 *    on the GPU (different streams or handles at the same time) race.  Each
 *    call writes every partial it later reads, so no clearing is needed.
 *  - The device address of the array is cached per device index for the
 *    life of the process; it does not survive cudaDeviceReset (or any other
 *    teardown of the device's primary context), after which this entry point
 *    must not be called again. */
#define MG_NOALLOC_MAX_PLANES 4096
mg_status mg_residual_norm_noalloc(mg_handle* h, const double* f, const double* x, double* out);

/* ---- kernel timing (opt-in, for benchmarks; not part of the method) ------
 * When enabled, every launch of a kernel class in class_mask (bit c = class c)
 * on a level in level_mask (bit l = level l) is bracketed by CUDA events on
 * the launching stream and its device time is accumulated per class and
 * level.  class_mask = 0 disables timing.  While a class run inside the
 * V-cycle (MG_K_CHEB_ZERO .. MG_K_BOTTOM, MG_K_DOT) is timed, the V-cycle is
 * launched kernel by kernel (not from the graph) so that the events are plain
 * stream events; timing only other classes keeps the graph.  Enabling or
 * disabling resets the counters. */
typedef enum {
  MG_K_CHEB_ZERO = 0,  /* smoother steps 0-1 from a zero guess (pre-smooth) */
  MG_K_CHEB_STEP = 1,  /* smoother step with a materialised iterate */
  MG_K_RESID = 2,      /* r = b - A x */
  MG_K_RESTRICT = 3,   /* full weighting (points = coarse points) */
  MG_K_PROLONG = 4,    /* x += P e */
  MG_K_BOTTOM = 5,     /* telescoped bottom levels + coarsest solve, one block or one cluster */
  MG_K_CG_DIR = 6,     /* p = z + beta p (float64) */
  MG_K_CG_UPD = 7,     /* x += alpha p, r -= alpha q, r.r (float64) */
  MG_K_DOT = 8,        /* rho = b.z, b the V-cycle's finest right-hand side (float64 accumulation), when
                          the V-cycle's last step does not form it */
  MG_K_CAST = 9,       /* float64 residual -> float32 V-cycle right-hand side */
  MG_K_CG_APPLY = 10,  /* q = A p, p.q with the float64 outer operator */
  MG_K_HOST_GAP = 11,  /* not a kernel: per outer CG iteration, the device time from the end of the
                          iteration's last kernel to the next V-cycle's launch, i.e. the read of the CG
                          scalars by the host, its convergence test and its next launch (points = 0) */
  MG_K_NCLASS = 12
} mg_kernel_class;
mg_status mg_timing_enable(mg_handle* h, int class_mask, int level_mask);
/* Totals for class cls on level l (0 = finest): device milliseconds, number of
 * launches and interior points processed (summed over launches). */
mg_status mg_timing_read(const mg_handle* h, int cls, int l, double* ms, long long* launches, double* points);

/* ---- float64 FMA throughput (measurement helper; not part of the method) --
 * The outer Krylov operator q = A p in float64 does eight float64 FMAs per
 * finest point against one neighbour load each, so on GPUs with a narrow
 * float64 pipe its bound is the float64 FMA rate, not memory bandwidth.  This
 * call times a kernel of independent FMA chains on the current device (8 per
 * thread, 4 blocks of 256 threads per SM, about 16 ms per launch on a GPU with
 * two float64 FMAs per clock per SM) on a stream of its own, one untimed launch
 * and then `launches` (1..100) launches timed with CUDA events, and writes the
 * fastest launch's rate to *tflops in TFLOP/s (one FMA = 2 flops).  The figure
 * is a lower bound on the float64 pipe's rate, not its peak: on GB300 it reads
 * about 0.84 of the nominal two FMAs per clock per SM, and long launches of the
 * float64 operator run faster than it.
 * Allocates and frees a small device buffer; synchronises its own stream.
 * Returns MG_ERR_ARG for launches outside 1..100 or a null tflops, MG_ERR_CUDA
 * if a CUDA call fails. */
mg_status mg_fp64_fma_peak(int launches, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
