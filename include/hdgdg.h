/*
 * hdgdg.h -- C ABI of the GB300 (sm_103a) IMEX HDG-DG shallow-water library.
 *
 * Method: Kang, Giraldo, Bui-Thanh, "IMEX HDG-DG: a coupled implicit hybridized
 * discontinuous Galerkin and explicit discontinuous Galerkin approach for shallow water
 * systems", arXiv:1711.02751.  The library advances the planar shallow-water system
 * (Sec. 3.1, eq. psweGov) on a periodic N x N uniform quadrilateral mesh of the unit
 * square with degree-k tensor-product Gauss-Lobatto nodes, by the IMEX HDG-DG scheme of
 * Algorithm 1 (Sec. 6): per stage, the explicit DG residual of the nonlinear flux
 * (eq. WeakForm_DG with the Rusanov flux, eq. Full_russanov / Linear_russanov), the
 * implicit HDG solve of the linear gravity-wave part (static condensation, eq.
 * linearizedHDGsystem_schur; global trace solve; local recovery, eq.
 * recover_volume_unknowns), and the stage combination (eq. hdgIMEXRK_qi / qn).
 *
 * Conventions shared by every entry point
 * -----------------------------------------
 * Mesh: element e = ey * N + ex; node n = j * (k+1) + i of an element, i along x, at GLL
 *   point xi_i: x = x0 + (ex + (1 + xi_i) / 2) h, y = x0 + (ey + (1 + xi_j) / 2) h, h = length/N.
 * Edges, periodic: edge r < N^2 is the right face of element r (normal +x); edge N^2 + r is
 *   the top face of element r (normal +y).  Walls: vertical edge ey*(N+1) + ix (ix = 0..N,
 *   normal +x) and horizontal edge N(N+1) + iy*N + ex (iy = 0..N, normal +y).  Trace vectors
 *   are [edge][field c][node b], b along the edge, fields (phi_hat, U_hat, V_hat).
 * User state: h (total depth), hu, hv as host arrays [n_el][(k+1)^2], double.
 * Internal state q = (phi_eta, U, V) = (g (h - B), g hu, g hv), B = H0 - b, phi_B = g B
 *   (Sec. 3, "phi = g H, U = phi u"); the row-level entry points take q as host arrays
 *   [3][n_el][(k+1)^2].
 * Ownership: the caller owns every host buffer it passes; the library copies in/out and
 *   owns all device memory it allocates.  A handle is not thread safe; distinct handles
 *   are independent.  All device work of a handle is issued on the stream given at
 *   create (the library makes its own non-blocking stream when NULL is given).
 * Errors: every call returns a status; on failure hdgdg_last_error(sim) holds a message.
 *   Entry points that return HDGDG_ECUDA leave the handle usable only for destroy.
 */
#ifndef HDGDG_H
#define HDGDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HDGDG_OK = 0,
    HDGDG_EINVAL = 1,          /* bad argument or unsupported configuration */
    HDGDG_ENOMEM = 2,          /* device or host allocation failed */
    HDGDG_ECUDA = 3,           /* a CUDA runtime call or kernel launch failed */
    HDGDG_ENOTCONVERGED = 4,   /* trace Krylov solve missed its tolerance within its cap */
    HDGDG_ENONFINITE = 5,      /* NaN or Inf in an input (or produced by a step) */
    HDGDG_ESTATE = 6           /* call made in the wrong order (e.g. step before set_state) */
} hdgdg_status;

/* Time integrators.  ARS2 / ARS3: the IMEX HDG-DG schemes of Sec. 6 (ARS(2,3,2), ARS(4,4,3)).
 * RK2 / RK3: the explicit RK DG schemes the paper compares against (Sec. 7.1, 7.2) -- the whole
 * flux with the Rusanov flux of eq. Full_russanov, advanced by Heun's method (RK2) or the
 * three-stage SSP method of Shu and Osher (RK3); no trace system is built for them, and the
 * implicit-stage row entry points return EINVAL. */
enum { HDGDG_ARS2 = 0, HDGDG_ARS3 = 1, HDGDG_RK2 = 2, HDGDG_RK3 = 3 };
/* Arithmetic of the path.
 * HDGDG_FP64:  every kernel in FP64.
 * HDGDG_MIXED: the trace Krylov solve runs as FP32 GMRES(m) cycles on an FP32 copy of the
 *              preconditioned trace matrix, each cycle restarted from the true residual
 *              g - S qhat computed in FP64 with the solution accumulated in FP64 (iterative
 *              refinement), and the DG residual of the nonlinear part is computed in FP32
 *              arithmetic on the FP64 state; residual norms, the stage combinations and mass
 *              sums stay in FP64.  The local condensation and recovery follow local_precision
 *              (FP64 unless another is chosen; HDGDG_LOCAL_F32X2 keeps them FP64-class on the
 *              FP32 pipes) and the refinement residual follows residual_f32x2.
 *              hdgdg_eval_nl always evaluates in FP64. */
enum { HDGDG_FP64 = 0, HDGDG_MIXED = 1 };
/* Arithmetic of the local condensation Z = A^{-1} R1 and recovery A^{-1} (tau qhat) (eq.
 * linearizedHDGsystem_schur, recover_volume_unknowns); implicit schemes only.
 * HDGDG_LOCAL_FP64: FP64 arithmetic (0, the default): A^{-1} applied through the Schur
 *                   complement on phi (see local_dense), or as the whole per-element FP64
 *                   A^{-1} with local_dense = 1.
 * HDGDG_LOCAL_FP32: a per-element FP32 copy of A^{-1}, FP32 products and sums (CUDA cores).
 * HDGDG_LOCAL_BF16: ONE operator shared by all elements -- a flat bottom (phi_B constant) and
 *                   one time step for all instances, else create fails with EINVAL -- applied
 *                   to all elements as one dense contraction on the tensor cores (tcgen05, BF16
 *                   inputs, FP32 accumulation in tensor memory).
 * HDGDG_LOCAL_F32X2: FP64-class on the FP32 pipes: the local operator (the Schur-complement
 *                   operators, or A^{-1} with local_dense = 1) held as FP32 pairs (hi + lo, 8
 *                   bytes per entry like FP64) and every row's dot product computed with the
 *                   compensated Dot2 scheme (exact products by FMA, TwoSum accumulation; Ogita,
 *                   Rump and Oishi 2005), about 1e-13 relative, at the HBM bound.
 * Vectors stay FP64 in every case; the precision variants of the paper's workloads report
 * their error against the FP64 form.
 * HDGDG_LOCAL_BF16_SPLIT: FP64-class on the tensor cores, for the same shared operator as
 *                   HDGDG_LOCAL_BF16 (flat bottom, one time step, k <= 4): every input row and
 *                   every operator column is scaled by a power of two and cut into five seven-bit
 *                   integer slices, exact in BF16 (the splitting of Ozaki, Ogita, Oishi and Rump,
 *                   Numer. Algorithms 2012); the slices' pairwise products with i + j < 5 run as
 *                   tcgen05 BF16 MMAs whose FP32 accumulators hold their sums exactly, and the
 *                   epilogue adds the five accumulators in 64-bit integers and scales in FP64:
 *                   about 35 bits, 3e-11 relative to the row and column scales.
 */
enum { HDGDG_LOCAL_FP64 = 0, HDGDG_LOCAL_FP32 = 1, HDGDG_LOCAL_BF16 = 2, HDGDG_LOCAL_F32X2 = 3,
       HDGDG_LOCAL_BF16_SPLIT = 4 };

typedef struct {
    int n_side;          /* N >= 2: elements per side of the periodic unit square */
    int degree_k;        /* polynomial degree k, 1 <= k <= 8 */
    double g;            /* gravitational acceleration (> 0) */
    double H0;           /* reference depth: B = H0 - b */
    int scheme;          /* HDGDG_ARS2, HDGDG_ARS3, HDGDG_RK2 or HDGDG_RK3 */
    double dt;           /* time step (> 0) */
    int precision;       /* HDGDG_FP64 or HDGDG_MIXED */
    double krylov_rtol;  /* GMRES stop: ||g - S qhat|| <= rtol ||g||; <= 0 selects 1e-15
                            (FP64) or 1e-9 (MIXED, FP64 residual of the refinement loop).
                            A restart cycle that fails to halve a true residual already below
                            1e-12 ||g|| ends the solve as converged (FP64 rounding floor). */
    int krylov_restart;  /* GMRES(m) restart length m <= 31; <= 0 selects 10 */
    int krylov_maxit;    /* cap on GMRES iterations per stage solve; <= 0 selects 2000 */
    int linear_only;     /* 1: drop NL (linear gravity-wave runs); 0: full method */
    int boundary;        /* HDGDG_PERIODIC (0), HDGDG_WALLS (1): reflecting walls on the four
                            sides (Sec. 4.3, eq. reflection; the trace condition becomes eq.
                            reflectionBC), or HDGDG_VORTEX (2): prescribed exact-solution
                            traces (below) */
    double x0;           /* domain [x0, x0 + length]^2 (node coordinates follow) */
    double length;       /* side of the square domain; <= 0 selects 1 */
    double bc_params[5]; /* HDGDG_VORTEX: beta, u_inf, v_inf, x_c, y_c of eq. tc_vortex_ic */
    int batch;           /* >= 1 (0 = 1): independent instances of this mesh advanced together;
                            every kernel covers all instances in one launch per stage and the
                            trace systems are solved as one block-diagonal system.  Arrays of
                            create / set_state / get_state are then [batch][n_el][(k+1)^2]. */
    const double* dt_per_instance; /* host [batch] time steps (read at create); NULL = dt for all */
    int local_precision; /* HDGDG_LOCAL_FP64 (0), HDGDG_LOCAL_FP32, HDGDG_LOCAL_BF16 or
                            HDGDG_LOCAL_F32X2 */
    int krylov_guess;    /* start of each implicit stage's trace solve: the polynomial extrapolation
                            in time of the same stage's solutions of the previous steps, of
                            order at most p = 1..6 (the last p solutions, x_0 = sum_{j=1..p}
                            (-1)^(j+1) C(p, j) x_{n-j}: 1 = x_{n-1}; 2 = 2 x_{n-1} - x_{n-2};
                            3: 3, -3, 1; ...), -1 = always start from zero, 0 selects 5.  Each
                            solve starts from the order <= p (or zero) whose residual is
                            smallest; one pass over g and the stored products S x_{n-j} (g - r
                            at the end of each solve) gives every candidate's residual, no
                            matrix product is needed.  The stop test stays
                            ||g - S qhat|| <= rtol ||g||. */
    int spmv_kernel;     /* FP32 trace-matrix product of the mixed form's inner cycles: 0 = one
                            thread per row component, neighbour vectors gathered through shared
                            memory; 1 = a persistent kernel that also streams the matrix through
                            shared memory with bulk (TMA) copies, two stages deep.  Identical
                            results (same summation order). */
    int krylov_ortho;    /* Gram-Schmidt of the mixed form's FP32 inner cycles: 0 = classical,
                            applied twice (CGS2; with the matrix-free operator the second pass
                            is delayed into the next Arnoldi step, whose product is taken of the
                            once-projected vector and corrected through the Arnoldi relation:
                            one pass over the basis fewer a step); 1 = classical, once.  The
                            FP64 form and the FP64 refinement residuals are not affected. */
    int residual_f32x2;  /* mixed form: 1 = the refinement's true residual g - S qhat in FP64-class
                            arithmetic on the FP32 pipes (S as an FP32 pair, compensated Dot2
                            sums, ~1e-13 relative; see HDGDG_LOCAL_F32X2); 0 = FP64. */
    int local_dense;     /* HDGDG_LOCAL_FP64 and HDGDG_LOCAL_F32X2: 0 (default) = A^{-1} applied
                            through the Schur complement on phi.  With collocated GLL nodes the
                            velocity blocks of A are diagonal, so U and V are eliminated node by
                            node and only the (phi, phi) block of A^{-1} ((k+1)^4 numbers per
                            element) is stored and read; the derivative couplings are rebuilt from
                            phi_B, tau and the GLL derivative matrix.  1 = the whole per-element
                            A^{-1} ((3 (k+1)^2)^2 numbers) as one dense product.  Same result up to
                            rounding.  The other local precisions are always dense. */
    int trace_operator;  /* how the mixed form's trace Krylov solve applies the preconditioned trace
                            matrix S M^{-1}: 0 = the assembled edge-block matrix (FP32 copy in the
                            inner cycles, FP32 pair in the refinement residual); 1 = matrix-free,
                            element by element: M^{-1} (block-Jacobi, held per edge as FP16 values
                            of the block scaled by a power of two -- the same numbers on every
                            path) edge by edge,
                            then per element the lift B, the Schur-complement local solve, C and D,
                            each edge row summed from its two elements' halves (FP32 in the inner
                            cycles, FP32 pairs in the refinement residual).  About 2.1 KB per element (k = 3) instead of
                            7.2 KB (FP32) or 14.3 KB (FP32 pair) of matrix.  1 needs precision =
                            HDGDG_MIXED with local_precision = HDGDG_LOCAL_F32X2 and local_dense = 0
                            (EINVAL otherwise); the FP64 form always uses the assembled matrix. */
    int host_steps;      /* 0 (default): each time step of an implicit scheme runs as ONE CUDA graph,
                            captured at the first step with a given configuration of the solver's
                            buffers (a handful of them, cached per handle) and replayed: the choice of
                            each trace solve's start, its restart cycles (a conditional while node)
                            and their stop tests run on the device, and the host waits once per step.
                            1: host-driven steps (the host waits for each restart cycle).  Steps run
                            host-driven anyway while the kernel-class timers are on and for
                            prescribed time-dependent boundary traces (HDGDG_VORTEX).  Same results
                            either way, bit for bit. */
    int dg_precision;    /* DG residual of the nonlinear part: 0 = the form's own (FP64 in HDGDG_FP64,
                            FP32 arithmetic in HDGDG_MIXED); 1 = BF16 inputs (the state, phi_B and
                            tau rounded to BF16) with FP32 arithmetic and accumulation -- the BF16
                            variant of the mixed form (HDGDG_MIXED and k <= 4 only, else EINVAL).
                            The residual is a nonlinear flux evaluation with P x P derivative
                            applications (P = k + 1 <= 5), not a dense contraction, so it runs on the
                            CUDA cores in every variant. */
    int krylov_guess_ls; /* 1 (HDGDG_MIXED only, krylov_guess >= 0): start each trace solve from the
                            least-squares projection on the affine span of the stored solutions --
                            the x_0 = sum_j alpha_j x_{n-j} (sum alpha = 1) whose residual
                            ||g - sum_j alpha_j S x_{n-j}|| is smallest, from one pass over g and
                            the stored products and a small solve -- or from zero when that is
                            smaller; every polynomial extrapolation of the same solutions is one
                            candidate of the projection.  0: the polynomial candidates (default). */
} hdgdg_config;

/* HDGDG_VORTEX: the exact-solution boundary conditions of the paper's moving-vortex test
 * (Sec. 7.1): every boundary trace is prescribed, qhat = q_exact(t) at the stage time, and the
 * DG flux sees q_exact(t) across the boundary; q_exact is eq. tc_vortex_ic with H_inf = H0 over
 * a flat bottom (b = 0), depth H_inf - beta^2/(16 pi^2 g) e^{-2(r^2-1)} (the printed
 * beta^2/(32 pi^2) at the paper's g = 2). */
enum { HDGDG_PERIODIC = 0, HDGDG_WALLS = 1, HDGDG_VORTEX = 2 };

typedef struct {
    long long steps;              /* time steps completed since set_state */
    long long krylov_iterations;  /* GMRES iterations summed over all stage solves */
    int last_krylov_iterations;   /* iterations of the most recent stage solve */
    double last_rel_residual;     /* ||g - S qhat|| / ||g|| of the most recent stage solve */
    double mass;                  /* sum_e J sum_ij w_i w_j phi_eta of the current state */
    long long kernel_launches;    /* CUDA kernels this handle launched in hdgdg_step since set_state */
    double time;                  /* simulated time since set_state (steps x dt) */
    int last_guess_order;         /* extrapolation order the most recent trace solve started from
                                     (0: zero start) */
    /* Meshes of >= 4096 elements: elements per block of the condensation and recovery kernels,
     * picked at create by timing each candidate tile on the handle's own operators -- the
     * Schur-complement kernels for degrees 2..4, the dense FP32-pair kernels for every degree
     * (0: the default tile, not tuned). */
    int local_tile_condense;
    int local_tile_recover;
    /* trace_operator = 1, meshes of >= 4096 elements, degrees 2..4: elements per block of the
     * matrix-free operator's element pass in the inner cycles and whether it loads the local
     * operator ahead of the traces (1) -- picked the same way (0, 0: the default, not tuned). */
    int trace_tile;
    int trace_tile_prefetch;
} hdgdg_stats;

/* Kernel classes of the per-kernel timers (hdgdg_kernel_time). */
enum {
    HDGDG_KT_SPMV = 0,      /* trace-matrix product of the Krylov loop (one kernel per launch) */
    HDGDG_KT_ORTHO = 1,     /* Gram-Schmidt dots, updates and normalisation of one iteration */
    HDGDG_KT_CONDENSE = 2,  /* A^{-1} R1 and the trace right-hand side */
    HDGDG_KT_RECOVER = 3,   /* local recovery of Q and L_i */
    HDGDG_KT_DG = 4,        /* DG residual of the nonlinear part */
    HDGDG_KT_COMBINE = 5,   /* stage combinations and the final update */
    HDGDG_KT_RESIDUAL = 6,  /* end of each restart cycle: the correction x += V y, the true residual
                               g - S x and its norm */
    HDGDG_KT_GUESS = 7,     /* initial guess of each trace solve: candidate residual norms, the
                               chosen extrapolation and residual, and the history update */
    HDGDG_KT_PRECOND = 8,   /* qhat = M^{-1} x~ after each trace solve (block-Jacobi blocks) */
    HDGDG_KT_COUNT = 9
};

typedef struct hdgdg_sim hdgdg_sim;

/* Device bytes the library will allocate for this configuration (for admission by
 * memory budget).  Returns 0 for an invalid configuration.  No GPU call is made. */
size_t hdgdg_bytes_required(const hdgdg_config* cfg);

/* GLL node coordinates x, y (host, [n_el][(k+1)^2] each) of one instance of the mesh of cfg,
 * in the node order above.  No GPU call is made.  EINVAL on a bad configuration or NULL. */
hdgdg_status hdgdg_node_coords(const hdgdg_config* cfg, double* x, double* y);

/* The library's degree-k Gauss-Lobatto-Legendre nodes and weights on [-1, 1] (host arrays of
 * k+1 doubles each), the collocation points of every element.  EINVAL if k is out of range. */
hdgdg_status hdgdg_gll(int degree_k, double* nodes, double* weights);

/* Build a simulation: mesh, GLL tables, the bottom phi_B = g (H0 - b), and the
 * time-invariant implicit-stage operators of Sec. 6 -- per-element A^{-1} and the
 * condensed trace matrix S = D - C A^{-1} B (eq. linearizedHDGsystem_schur), assembled
 * once into edge-block CSR with its block-Jacobi preconditioner folded in (the
 * operators are the same for every stage and step because the implicit diagonal is
 * constant, Sec. 7.1).  bottom_b: host [n_el][(k+1)^2] (NULL = flat, b = 0).
 * cuda_stream: a cudaStream_t to issue work on, or NULL.  On success *out owns the
 * handle; release it with hdgdg_destroy.  Fails with EINVAL, ENOMEM, ENONFINITE or ECUDA;
 * when the failure happens after the handle exists, *out still receives it so that
 * hdgdg_last_error can explain the failure -- its only other valid use is hdgdg_destroy. */
hdgdg_status hdgdg_create(const hdgdg_config* cfg, const double* bottom_b, void* cuda_stream,
                          hdgdg_sim** out);

/* Copy a user state (host arrays h, hu, hv [n_el][(k+1)^2]) in and start a new trajectory:
 * step counters, simulated time and the trace solve's initial-guess history are reset.
 * ENONFINITE if any value is not finite or h - B leaves phi = g h <= 0. */
hdgdg_status hdgdg_set_state(hdgdg_sim* sim, const double* h, const double* hu, const double* hv);

/* Replace the state of a running trajectory (e.g. a host that corrects the state between
 * steps; the paper has no counterpart): like hdgdg_set_state, but the step counters, the
 * simulated time and the initial-guess history are kept.  Arrays as hdgdg_set_state, copied
 * in.  ESTATE before the first hdgdg_set_state; ENONFINITE as hdgdg_set_state (the previous
 * state is then kept). */
hdgdg_status hdgdg_update_state(hdgdg_sim* sim, const double* h, const double* hu, const double* hv);

/* Advance n_steps >= 0 time steps of Algorithm 1.  Synchronises the stream on return.
 * ENOTCONVERGED if a trace solve misses krylov_rtol within krylov_maxit (the state is
 * left at the last completed step); ENONFINITE if a step produced NaN/Inf (state left at
 * the last finite step); ESTATE before set_state. */
hdgdg_status hdgdg_step(hdgdg_sim* sim, int n_steps);

/* Copy the current state out to host arrays h, hu, hv [n_el][(k+1)^2]. */
hdgdg_status hdgdg_get_state(hdgdg_sim* sim, double* h, double* hu, double* hv);

/* Counters of the run so far; computes the mass of the current state on the device. */
hdgdg_status hdgdg_get_stats(hdgdg_sim* sim, hdgdg_stats* out);

/* Checkpoint / resume (the paper has no counterpart; long runs and preempted serving
 * requests).  A checkpoint holds the state, the simulated time, the counters and the trace
 * solve's initial-guess history, so that a handle created with the same configuration and
 * bottom, loaded from it, continues bit for bit as the uninterrupted run.  The layout is this
 * library version's, host byte order.  hdgdg_checkpoint_bytes: the size a checkpoint of the
 * current state needs (0 before set_state).  hdgdg_save_checkpoint copies it into the caller's
 * host buffer buf of `bytes` (EINVAL if too small, ESTATE before set_state).
 * hdgdg_load_checkpoint replaces the handle's state and history from buf; EINVAL if buf is not a
 * checkpoint, is truncated, or was taken with another mesh, degree, scheme, arithmetic,
 * boundary, batch, time step (per-instance time steps included), g, H0 or domain.  The bottom is not recorded: pass the same bottom
 * to hdgdg_create. */
size_t hdgdg_checkpoint_bytes(hdgdg_sim* sim);
hdgdg_status hdgdg_save_checkpoint(hdgdg_sim* sim, void* buf, size_t bytes);
hdgdg_status hdgdg_load_checkpoint(hdgdg_sim* sim, const void* buf, size_t bytes);

/* Message of the last failure on this handle ("" if none; a static message if sim is NULL). */
const char* hdgdg_last_error(const hdgdg_sim* sim);

/* Release every device and host resource of the handle (NULL is a no-op). */
void hdgdg_destroy(hdgdg_sim* sim);

/* ---- row-level entry points (one step of the hot path each; host buffers) ----------
 * Prescribed boundary data (HDGDG_VORTEX) are taken at the handle's current time (0 after
 * create or set_state, then steps x dt). */

/* M^{-1} NL(q) of Sec. 4.3 (DG volume term plus Rusanov face terms of the nonlinear
 * flux F_NL = F - F_L) for the internal state q [3][n_el][(k+1)^2]; out has the same
 * layout.  The bottom is the handle's. */
hdgdg_status hdgdg_eval_nl(hdgdg_sim* sim, const double* q, double* out);

/* Right-hand side of the condensed trace system for stage data R1 [3][n_el][(k+1)^2]:
 * g = -C A^{-1} R1 (eq. linearizedHDGsystem_schur with R2 = 0), one conservation row per
 * trace node in POINTWISE form, i.e. eq. HDGcont divided by the positive face quadrature
 * weight (h/2) w_b of the node.  out: [edge][c][b]. */
hdgdg_status hdgdg_condense_rhs(hdgdg_sim* sim, const double* R1, double* out);

/* y = S x for the condensed trace matrix S = D - C A^{-1} B in the pointwise row scaling
 * of hdgdg_condense_rhs.  x, y: [edge][c][b]. */
hdgdg_status hdgdg_trace_apply(hdgdg_sim* sim, const double* x, double* y);

/* Select the tile of the matrix-free operator's element pass in the inner Krylov cycles
 * (trace_operator = 1), overriding the one picked at create: 0 the default; 1..8 (degrees
 * 2..4) blocks of 128, 256 or 512 threads, with or without the local operator's row loaded into
 * registers ahead of the traces, under different register caps.  Every tile gives the same
 * result bit for bit.  Cached step graphs are dropped.  HDGDG_EINVAL when the handle has no such
 * pass or the tile is not available. */
hdgdg_status hdgdg_set_trace_tile(hdgdg_sim* sim, int tile);

/* Select the tiles of the Schur-complement condensation and recovery kernels (local solves
 * through the Schur complement on phi), overriding the ones picked at create: 0 the default;
 * 1, 2 (degrees 2..4) blocks of 128 or 512 threads; 3 (degree 3) 128 threads with the element
 * operators staged in shared memory by bulk asynchronous copies.  Every tile gives the same
 * result bit for bit.  Cached step graphs are dropped.  HDGDG_EINVAL when the handle's local
 * solves are not these kernels or a tile is not available. */
hdgdg_status hdgdg_set_local_tiles(hdgdg_sim* sim, int condense_tile, int recover_tile);

/* One implicit stage solve (Algorithm 1, the "else" branch): condense, GMRES on the trace
 * system, recover Q = A^{-1}(R1 - B qhat).  R1, Q: [3][n_el][(k+1)^2]; qhat: [edge][c][b]
 * (may be NULL).  *iterations (may be NULL) receives the GMRES iteration count. */
hdgdg_status hdgdg_stage_solve(hdgdg_sim* sim, const double* R1, double* Q, double* qhat,
                               int* iterations);

/* ---- measurement helpers --------------------------------------------------------- */

/* Switch the per-kernel-class timers on (1) or off (0) and zero them.  When on, the
 * library brackets each timed launch group with CUDA events on the handle's stream and
 * accumulates their elapsed times; timing adds two event records per group. */
hdgdg_status hdgdg_set_kernel_timing(hdgdg_sim* sim, int on);

/* Accumulated device time (ms) and number of timed launch groups of kernel class cls
 * (HDGDG_KT_*) since the timers were last switched on.  EINVAL for a bad class. */
hdgdg_status hdgdg_kernel_time(hdgdg_sim* sim, int cls, double* total_ms, long long* launches);

/* Measured FP64 fused-multiply-add throughput of the current device in TFLOP/s (2 flops
 * per FMA), from a register-resident FMA chain kernel timed with CUDA events.  Used as
 * the denominator of ALU-bound roofline fractions.  ECUDA on failure. */
hdgdg_status hdgdg_measure_fp64_tflops(double* tflops);

/* Measured FP64 <-> FP32 conversion throughput of the current device (conversions per second),
 * from chain kernels timed with CUDA events: *hardware_per_s with the conversion instructions the
 * compiler emits for casts, *integer_per_s with the library's integer-pipe routines (the mixed
 * and FP32-pair kernels use the latter; on GB300 the former run at the FP64 rate).  ECUDA on
 * failure, EINVAL for NULL. */
hdgdg_status hdgdg_measure_conversion_rates(double* hardware_per_s, double* integer_per_s);

/* ---- uneven ensembles ------------------------------------------------------------------------
 * Many independent instances of different mesh sizes and degrees advanced together (the
 * batched-ensemble workload; the paper runs one instance at a time).  Members sharing (N, k)
 * form a group; every geometry-dependent kernel of a time step -- the DG residual, the
 * condensation, the matrix-free trace operator's passes, the recovery -- runs as ONE persistent
 * launch over all groups, walking a device work list of (group, block) items, and the stage
 * combinations and Krylov vector operations cover the whole ensemble as one vector; each time step
 * is one replayed CUDA graph (see host_steps).  The members' trace systems form one
 * block-diagonal system solved by one GMRES whose stop test is on the whole ensemble's residual,
 * so a member's result agrees with its lone run to the solver tolerance, not bit for bit.
 * base: the shared configuration (g, H0, scheme ARS2 or ARS3, Krylov options, guess order); it
 * must select the mixed form with FP32-pair local solves and the matrix-free trace operator
 * (precision = HDGDG_MIXED, local_precision = HDGDG_LOCAL_F32X2, trace_operator = 1), a periodic
 * boundary and the full method (linear_only = 0); its n_side, degree_k, dt, batch are ignored.
 * Member m: n_side[m] >= 2, 2 <= degree_k[m] <= 4, its own time step dt[m] > 0 and bottom
 * bottom_b[m] (host [N^2][(k+1)^2]; bottom_b or an entry may be NULL = flat); at most 32 distinct
 * (N, k).  States are host arrays [N^2][(k+1)^2] per member as for hdgdg_set_state.
 * set_state of any member drops the ensemble's solver history (the next solves start from zero)
 * and restarts its counters; step advances every member by n_steps of its own time step.  Errors
 * as for the lone handle; EINVAL for a configuration outside the above. */
typedef struct hdgdg_ensemble hdgdg_ensemble;
hdgdg_status hdgdg_ensemble_create(const hdgdg_config* base, int n_members, const int* n_side, const int* degree_k,
                                   const double* dt, const double* const* bottom_b, void* cuda_stream,
                                   hdgdg_ensemble** out);
hdgdg_status hdgdg_ensemble_set_state(hdgdg_ensemble* ens, int member, const double* h, const double* hu,
                                      const double* hv);
hdgdg_status hdgdg_ensemble_step(hdgdg_ensemble* ens, int n_steps);
hdgdg_status hdgdg_ensemble_get_state(hdgdg_ensemble* ens, int member, double* h, double* hu, double* hv);
/* Counters of the whole ensemble (its mass field is 0: per-member masses follow from get_state). */
hdgdg_status hdgdg_ensemble_get_stats(hdgdg_ensemble* ens, hdgdg_stats* out);
const char* hdgdg_ensemble_last_error(const hdgdg_ensemble* ens);
void hdgdg_ensemble_destroy(hdgdg_ensemble* ens);

/* ---- allocation-free entry point ------------------------------------------------- */

/* Mass sum_e J sum_ij w_i w_j phi_eta of ONE instance's state -- the mass hdgdg_get_stats
 * reports for a handle of batch 1 -- for callers that cannot allocate device memory: code that
 * runs inside another framework's fixed memory pool, a real-time loop that must stay out of the
 * CUDA allocator, or a host callback, none of which may call cudaMalloc.  The paper has no
 * counterpart: it is a service of this library.
 * n_side: elements per side N of the square mesh (n_side * n_side elements, any boundary);
 * length: side of the square domain, as hdgdg_config.length (<= 0 selects 1), which sets the
 * element Jacobian J = (length / (2 N))^2.  For a batched handle, call once per instance on that
 * instance's slice and add the results.
 * d_phi_eta: device array [n_el][(k+1)^2] (phi_eta = g (h - B)); d_mass: one device double,
 * written on the given stream (NULL = legacy default stream); both belong to the caller.
 * The per-element partial sums live in a fixed array of the library's static device memory
 * (8 MiB on every GPU that loads the library, held until the process exits), so the call
 * allocates nothing.  Each call looks the array's address up in the current context; the first
 * call on a device may load the library's device code, so it should come before any stream
 * capture.  The array is shared by all calls on a device and keeps the last call's contents;
 * calls that overlap on the GPU race on it, so issue them on one stream or serialise them.
 * EINVAL for n_side * n_side > 2^20 elements (the array's capacity), n_side < 1, a bad degree, a
 * non-finite length or NULL pointers; ECUDA if the lookup or a launch fails. */
hdgdg_status hdgdg_mass_noalloc(int n_side, int degree_k, double length, const double* d_phi_eta,
                                double* d_mass, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HDGDG_H */
