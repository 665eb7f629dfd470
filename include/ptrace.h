/*
 * ptrace.h -- C ABI of the GB300 library for the displacement-probed
 * estimator of Tr(P A^{-1}) on 4D toroidal lattices.
 *
 * Method: Switzer, Stathopoulos, Romero, Laeuchli, Orginos, "Probing for the
 * trace estimation of a permuted matrix inverse corresponding to a lattice
 * displacement" (arXiv 2106.01275).  Each entry point cites the passage
 * that defines the operation it performs.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: PT_OK (0) or a negative PT_ERR_* code.  After an error,
 *   pt_last_error() returns a one-line message (thread-local).
 * - Lattice: dims[4] = (D_0, D_1, D_2, D_3) = (x, y, z, t).  Sites are stored
 *   in the order idx = x_0 + D_0 (x_1 + D_1 (x_2 + D_2 x_3)), x_0 fastest;
 *   N = D_0 D_1 D_2 D_3.  Every D_i >= 1 (the kernels take any size, no
 *   power-of-two or tile-multiple requirement).
 * - Displacement (Sec. 3): P is the permutation (P f)(x) = f(x + p e_mu) with
 *   periodic wrap and no boundary sign, so Tr(P A^{-1}) = sum_x A^{-1}(x+p, x).
 * - Fields in the ABI layout ("user layout"), all on the device:
 *     scalar (Laplacian, dof 1): float64 [nrhs][N]
 *     spinor (Wilson, dof 12):   complex128 [nrhs][N][4 spin][3 colour],
 *                                interleaved (re, im); component a = 3 spin + colour
 *     links:                     complex128 [N][4 mu][3][3] (row, column)
 * - Ownership: the caller allocates and frees every buffer whose pointer it
 *   passes.  A context owns its work space (device memory, streams, graphs);
 *   an operator owns its packed copy of the links.  Pointers marked "host"
 *   are host memory; all others are device memory of the context's device.
 * - Streams: work is enqueued on the context's stream.  Entry points that
 *   return host results synchronise that stream before returning; the others
 *   are asynchronous with respect to the host.
 * - Contexts are not thread-safe: one host thread per context at a time.
 */
#ifndef PTRACE_H
#define PTRACE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PT_API __attribute__((visibility("default")))
#else
#define PT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PT_OK            0
#define PT_ERR_ARG      (-1)  /* invalid argument (size, pointer, mode)            */
#define PT_ERR_CUDA     (-2)  /* a CUDA runtime call failed                        */
#define PT_ERR_NOCONV   (-3)  /* a solve did not reach tol within maxit            */
#define PT_ERR_TIMEOUT  (-4)  /* a bounded device wait or host loop gave up        */
#define PT_ERR_NUMERIC  (-5)  /* NaN/Inf or a Krylov breakdown (zero denominator)  */
#define PT_ERR_OOM      (-6)  /* device allocation of the work space failed        */

/* ---- precision modes of the solver ---- */
#define PT_PREC_FP64        0 /* all vectors and arithmetic FP64                     */
#define PT_PREC_MIXED_FP32  1 /* FP32 inner Krylov inside FP64 defect correction      */
#define PT_PREC_MIXED_BF16  2 /* as MIXED_FP32, inner vectors stored in BF16          */

/* ---- noise and visit orders ---- */
#define PT_NOISE_Z2        0  /* +-1            (Sec. 1, Rademacher)                 */
#define PT_NOISE_Z4        1  /* +-1, +-i       (Sec. 1, complex case)               */
#define PT_ORDER_NATURAL   0  /* storage order (Sec. 3.1)                            */
#define PT_ORDER_REDBLACK  1  /* even-parity sites, then odd, each in storage order   */

typedef struct pt_ctx pt_ctx;
typedef struct pt_op pt_op;

/* Solver statistics of one pt_solve / pt_trace_PAinv / pt_grad call. */
typedef struct pt_stats {
    int64_t n_rhs;            /* right-hand sides solved                                 */
    int64_t inner_iters;      /* Krylov iterations summed over right-hand sides          */
    int64_t outer_iters;      /* FP64 true-residual evaluations summed over RHS          */
    int64_t site_rhs_applies; /* operator applications x sites, summed over RHS          */
    int64_t engine_iters;     /* batched engine iterations (each = one graph body)       */
    int64_t graph_launches;   /* CUDA graph launches                                    */
    int64_t kernel_launches;  /* kernels launched by the library in this call           */
    double  max_relres;       /* largest final FP64 true relative residual               */
    int32_t n_slots;          /* right-hand sides resident at once                      */
    int32_t n_noconv;         /* right-hand sides that hit maxit                         */
} pt_stats;

/* ------------------------------------------------------------------ context */

/* Library version (major*10000 + minor*100 + patch). */
PT_API int pt_version(void);

/* Copy the calling thread's last error message into buf (always NUL-terminated). */
PT_API int pt_last_error(char *buf, size_t n);

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t to
 * enqueue on, or NULL for a library-owned non-blocking stream (to use the
 * legacy default stream pass cudaStreamLegacy, i.e. (void *)0x1).  *ctx
 * receives the handle (NULL on failure). */
PT_API int pt_create(pt_ctx **ctx, int device, void *stream);

/* Release the context, its work space, graphs and (if owned) stream. */
PT_API int pt_destroy(pt_ctx *ctx);

/* Block until all work enqueued by the context has finished. */
PT_API int pt_synchronize(pt_ctx *ctx);

/* Cap on the device bytes the solver engine may hold for resident
 * right-hand sides (default 16 GiB).  Larger budgets keep more RHS in flight. */
PT_API int pt_set_memory_budget(pt_ctx *ctx, size_t bytes);

/* Cap on the right-hand sides the solver engine keeps in flight (0 = no cap
 * beyond the memory budget).  n = 1 gives the plain one-RHS-at-a-time solve. */
PT_API int pt_set_max_slots(pt_ctx *ctx, int n);

/* Cap on the CUDA-graph launches of one solver-engine run (a host-side
 * watchdog for callers with a time budget; 0 = the engine's own bound, which
 * every run meets: maxit Krylov iterations per right-hand side plus a margin
 * per outer restart and per retire/refill).  A run that reaches the cap stops
 * between two graph launches, with nothing left in flight, and returns
 * PT_ERR_TIMEOUT; the context stays usable. */
PT_API int pt_set_launch_limit(pt_ctx *ctx, int64_t n);

/* Free parameters of the solver engine (not in the paper).
 *   delta        inner relative tolerance of a mixed-precision Krylov cycle
 *                (0 for FP64: the inner solve runs to the outer tolerance)
 *   group        right-hand sides whose work items are interleaved site block
 *                by site block, so that they share the links through L2
 *   graph_iters  engine iterations captured in one CUDA graph (host polls
 *                the completion flag once per graph launch)
 *   rhs_block    right-hand sides per work item of the Wilson applies: 1;
 *                2 on the full system in mixed precision (each link load
 *                serves two right-hand sides); 8 in even-odd mode with
 *                256-thread CTAs (a work item covers 256 sites for eight
 *                slots, one warp each, and stages the links of every 32 sites
 *                once in shared memory for all eight); other combinations
 *                fall back to 1; 0 means 1
 *   overlap      1: within an engine iteration the contraction and the FP64
 *                outer steps run as CUDA-graph branches beside the inner
 *                Krylov kernels (they work on disjoint right-hand sides);
 *                0: one kernel after another
 *   evenodd      every lattice side even: 1 solves each right-hand side
 *                through the Schur complement on the even sites, with the
 *                odd half rebuilt from it (Laplacian S = d - H_eo H_oe / d,
 *                d = 8 + m2, H the hops, x_o = (b_o + H_oe x_e) / d; Wilson
 *                S = 1 - kappa^2 D_eo D_oe, x_o = b_o + kappa D_oe x_e); the
 *                stopping test stays the full system's ||b - A x|| / ||b||.
 *                0: the full system.  The default is 1 where allowed; it is
 *                ignored for odd sides and by pt_grad, and it replaces
 *                rhs_block by 1.
 *   cta_threads  threads of every work-item kernel's CTA: 64, 128 or 256
 *                (0 means 256)
 *   sites_per_thread  Laplacian: lattice sites (even-odd: half-lattice
 *                entries) per thread of a work item: 4, 8 or 16 (0 means 8);
 *                a work item is cta_threads x sites_per_thread sites.  The
 *                Wilson kernels take one site per thread (pt_get_tuning
 *                reports 1).
 * seconds_per_rhs is an output of pt_autotune (device time per trial RHS). */
typedef struct pt_tune {
    double delta;
    int32_t group;
    int32_t graph_iters;
    int32_t rhs_block;
    int32_t overlap;
    int32_t evenodd;
    int32_t cta_threads;
    int32_t sites_per_thread;
    double seconds_per_rhs;
} pt_tune;

/* Autotuner: solves the same trial right-hand sides (up to trial_rhs probes
 * of one noise set spread over the colours of col_dev) with candidate
 * parameters, by coordinate descent over evenodd (every side even),
 * delta (mixed precision), rhs_block and group (Wilson), the work-item shape
 * (cta_threads; sites_per_thread for the Laplacian) and graph_iters
 * (overlap stays as set), keeps the fastest, and stores it in the context
 * for this operator's (kind, precision, lattice); later solves, traces and
 * gradients with that key use it.  *best (host) receives it.  Synchronises. */
PT_API int pt_autotune(pt_ctx *ctx, const pt_op *op, const int32_t *col_dev, int n_colours, int mu, int noise,
                       uint64_t seed, int prec, double tol, int maxit, int trial_rhs, pt_tune *best);

/* Install tuning parameters for (op kind, prec, lattice), e.g. from a cache;
 * t = NULL restores the defaults.  pt_get_tuning returns the parameters the
 * next run with that key will use. */
PT_API int pt_set_tuning(pt_ctx *ctx, const pt_op *op, int prec, const pt_tune *t);
PT_API int pt_get_tuning(pt_ctx *ctx, const pt_op *op, int prec, pt_tune *t);

/* Enable (1) or disable (0) per-kernel CUDA-event timing inside the engine.
 * pt_profile_read returns, for the kernel class `which` (0 = the operator
 * apply of the inner Krylov iteration), the launches and the summed
 * device milliseconds since the last reset. */
PT_API int pt_profile_enable(pt_ctx *ctx, int on);
PT_API int pt_profile_read(pt_ctx *ctx, int which, int64_t *launches, double *ms, int reset);

/* ---------------------------------------------------------------- operators */

/* Shifted scalar Laplacian, periodic in all four dimensions:
 *   (A f)(x) = (8 + m2) f(x) - sum_mu [ f(x + mu) + f(x - mu) ].
 * The paper abstracts its operator to a non-singular lattice matrix (Sec. 2);
 * this is the scalar instance used for its Fig. 1 and Fig. 2 examples. */
PT_API int pt_op_laplacian(pt_ctx *ctx, const int dims[4], double m2, pt_op **op);

/* Wilson-Dirac operator (the LQCD operator family of Sec. 4.2, without the
 * clover term):
 *   (A psi)(x) = psi(x) - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x + mu) eta
 *                                       + (1 + g_mu) U_mu(x - mu)^+ psi(x - mu) eta ]
 * chiral Euclidean gamma basis g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0,1],[1,0]];
 * eta = -1 on hops across the t boundary when antiperiodic_t, else +1.
 * U_dev: links in the user layout (device, read once; the operator keeps a
 * packed FP64 and FP32 copy, so the caller may free U_dev afterwards). */
PT_API int pt_op_wilson(pt_ctx *ctx, const int dims[4], const double *U_dev, double kappa,
                 int antiperiodic_t, pt_op **op);

/* Degrees of freedom per site of the operator (1 or 12), or a negative error. */
PT_API int pt_op_dof(const pt_op *op);

/* Free an operator (its packed links).  Waits for the device.  It does not
 * use the context, so it may be called before or after pt_destroy of the
 * context the operator was made with (e.g. by a garbage collector that
 * finalises both in no particular order). */
PT_API int pt_op_destroy(pt_op *op);

/* y = A x for nrhs fields in the user layout (device).  prec: PT_PREC_FP64
 * applies in FP64; PT_PREC_MIXED_FP32 rounds x to FP32, applies the FP32
 * kernel of the inner solver and widens the result; PT_PREC_MIXED_BF16 rounds
 * x to BF16 storage first.  x and y must not overlap. */
PT_API int pt_apply(pt_ctx *ctx, const pt_op *op, const double *x_dev, double *y_dev, int nrhs, int prec);

/* ---------------------------------------------------------------- colouring */

/* Host-side stencil of the displaced distance-k neighbourhood (Eq. (8), and
 * the union over several displacements of Sec. 3.4):
 *   O = { o != 0 : ||o - p_n e_mu||_1 <= k  or  ||o + p_n e_mu||_1 <= k, some n }
 * sorted lexicographically in (o_0, o_1, o_2, o_3).  offsets_out (host) receives
 * up to max_offsets rows of 4 ints; *n_offsets the full count.  Returns
 * PT_ERR_ARG if max_offsets is too small (after writing *n_offsets). */
PT_API int pt_stencil(int mu, const int *p_list, int n_p, int k, int *offsets_out, int max_offsets,
               int *n_offsets);

/* Greedy displaced distance-k colouring (Algorithm 1, Sec. 3.1): nodes are
 * visited in `order`; each takes the smallest colour (0-based) not held by an
 * already coloured node of N(x, p, k) (x itself excluded).  Bit-exact with the
 * sequential definition.  col_dev: int32 [N] (device, written); *n_colours
 * (host) receives m.  Synchronises the context stream. */
PT_API int pt_colour(pt_ctx *ctx, const int dims[4], int mu, const int *p_list, int n_p, int k,
              int order, int32_t *col_dev, int *n_colours);

/* Nested ("hierarchical") colouring: a colouring at distance k grown from a
 * coarser one (the paper leaves hierarchical probing of displaced colourings
 * to its Sec. 2.3 discussion; this is the reading used for a colouring grown
 * from k1 to k > k1).  The greedy walk of pt_colour in which a node only
 * sees the neighbours of N(x, p, k) that share its parent colour
 * parent_dev[x]; the colour of x is the pair (parent colour, local first-fit
 * colour), the pairs numbered 0, 1, ... in the order the walk first meets
 * them.  Nodes with the same colour share the parent colour, so every parent
 * class is a union of classes, and no two neighbours share a colour.
 * parent_dev: int32 [N] (device, read) with values in [0, n_parent)
 * (PT_ERR_ARG otherwise); col_dev: int32 [N] (device, written); *n_colours
 * (host).  With a constant parent the result is pt_colour's.  Uses a
 * temporary stream-ordered allocation; synchronises the context stream. */
PT_API int pt_colour_nested(pt_ctx *ctx, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                            const int32_t *parent_dev, int n_parent, int32_t *col_dev, int *n_colours);

/* Count ordered pairs (x, y), y in N(x,p,k), y != x, with equal colours: zero
 * for a valid colouring (Sec. 3.1).  *n_conflicts is host.  Synchronises. */
PT_API int pt_colour_conflicts(pt_ctx *ctx, const int dims[4], int mu, const int *p_list, int n_p,
                        int k, const int32_t *col_dev, int64_t *n_conflicts);

/* Allocation-free form of pt_colour_conflicts (the paper has no counterpart:
 * this is a service for callers that cannot allocate device memory, such as
 * a host program whose own pool allocator owns the device memory, a caller
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree,
 * or one running under a fixed device-memory cap).  Same result as
 * pt_colour_conflicts, without a context: it runs on the calling thread's
 * current device and on `stream` (a cudaStream_t; NULL = the default stream).
 * Scratch is a file-scope device array of the library: at most 16384 distinct
 * stencil offsets after repeats from overlapping displacements are merged
 * (larger stencils return PT_ERR_ARG) and one counter, 256 KiB in
 * total, held by every device that loads the library until the process
 * exits.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Calls neither allocate nor free device memory.  Every call shares the
 * array, which keeps the last call's contents; the call clears its counter
 * itself.  Calls are serialised inside the process and each one finishes on
 * the GPU before it returns; work that another caller enqueues to use this
 * array concurrently would race with it.  *n_conflicts is host.
 * Synchronises `stream`. */
PT_API int pt_colour_conflicts_noalloc(void *stream, const int dims[4], int mu, const int *p_list, int n_p,
                                       int k, const int32_t *col_dev, int64_t *n_conflicts);

/* ------------------------------------------------------------------ tiles */

/* Tile of Sec. 3.5 for a (p_list, k)-colouring of the lattice `dims`
 * (host-only, no GPU needed).  A tile holds a whole neighbourhood: every side
 * at least 2k + 1, the side along mu at least 2(max p + k) + 1.  Its sides
 * divide the lattice's: each is the smallest divisor of the lattice side at
 * or above the minimum (the smallest power of two above it on power-of-two
 * lattices, as in Table 2), else the lattice side.  tile_out: 4 ints (host).
 * PT_ERR_ARG on a NULL pointer, mu outside 0..3, k outside 0..64, n_p outside
 * 1..64 or p outside 0..4096. */
PT_API int pt_tile_dims(const int dims[4], int mu, const int *p_list, int n_p, int k, int tile_out[4]);

/* Repeat a tile's colouring over the lattice (Sec. 3.5):
 * col[x] = tile_col[x mod tile_dims].  tile_col_dev: int32 [prod tile_dims]
 * (device, read); col_dev: int32 [prod dims] (device, written); the two must
 * not overlap.  Every tile side must divide the lattice side (PT_ERR_ARG).
 * Asynchronous on the context stream. */
PT_API int pt_tile_replicate(pt_ctx *ctx, const int tile_dims[4], const int32_t *tile_col_dev, const int dims[4],
                             int32_t *col_dev);

/* pt_colour on the tile of pt_tile_dims, repeated over the lattice by
 * pt_tile_replicate.  col_dev: int32 [N] of the lattice (device, written);
 * *n_colours (host): the tile's colour count; tile_out (host, 4 ints): the
 * tile used.  The tile's colours live in a temporary device buffer
 * (stream-ordered allocation, freed before returning).  Synchronises the
 * context stream. */
PT_API int pt_colour_tiled(pt_ctx *ctx, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                           int32_t *col_dev, int *n_colours, int tile_out[4]);

/* Clearance of a colouring at other displacements (Thm 3.6; Sec. 4.3, Table
 * 5).  For every displacement p = p_list[i] along mu and distance
 * k = k_list[j], the shell S_x(p, k) is the set of nodes y != x of the torus
 * whose L1 distance to the nearer of x + p e_mu and x - p e_mu is exactly k
 * (each node counted once).  Outputs (host, int64 [n_p][n_k], row i = p):
 *   matches_out[i][j] = sum over x of #{y in S_x(p, k) : col(y) = col(x)},
 *   shell_out[i][j]   = |S_x(p, k)| (the same for every x).
 * The average percentage of uncleared neighbours printed in Table 5 is
 * 100 matches / (N |S|).  col_dev: int32 [N] (device, read).  Lattice sides
 * 1..65535, 1 <= n_p, n_k <= 64, p in 0..4096, k in 0..32; all distinct
 * offsets of the requested shells together at most 524,280.  Synchronises
 * the context stream. */
PT_API int pt_clearance(pt_ctx *ctx, const int dims[4], int mu, const int32_t *col_dev, const int *p_list, int n_p,
                        const int *k_list, int n_k, int64_t *matches_out, int64_t *shell_out);

/* ------------------------------------------------------------------- probes */

/* Materialise one probing vector (Eq. (4) with the noise of Eq. (5) and the
 * spin-colour dilution of Sec. 4.2):
 *   v(x, b) = z0_set(x) [col(x) = colour] delta_{b, component}
 * z0 from SplitMix64: h = mix64(key + (x+1) G), key = mix64(seed + (set+1) G),
 * G = 0x9E3779B97F4A7C15; Z2: 1 - 2 (h >> 63); Z4: i^(h >> 62).
 * dof 1 -> v_dev float64 [N] (Z2 only); dof 12 -> complex128 [N][12].
 * The solver regenerates probes in-kernel; this call exists for checks. */
PT_API int pt_make_probes(pt_ctx *ctx, const int32_t *col_dev, int64_t N, int colour, int noise,
                   uint64_t seed, int set, int dof, int component, double *v_dev);

/* ------------------------------------------------------------------ solves */

/* Solve A X = B for nrhs right-hand sides in the user layout (device; X is
 * written, initial guess zero).  Stops each RHS when its FP64 true relative
 * residual ||b - A x|| / ||b|| < tol.  Laplacian: CG; Wilson: BiCGStab.
 * Mixed modes run the Krylov iteration in FP32 (or BF16 storage) inside an
 * FP64 defect-correction loop.  iters_out / relres_out: host arrays [nrhs]
 * or NULL.  stats: host or NULL.  Returns PT_ERR_NOCONV if any RHS hit maxit
 * (X still holds its last iterate).  Synchronises. */
PT_API int pt_solve(pt_ctx *ctx, const pt_op *op, const double *B_dev, double *X_dev, int nrhs,
             int prec, double tol, int maxit, int *iters_out, double *relres_out, pt_stats *stats);

/* ------------------------------------------------------------------ traces */

/* Probed estimates of Tr(P_n A^{-1}) for every displacement p_list[n] along mu
 * (Eqs. (1), (4), (5), spin-colour dilution of Sec. 4.2):
 *   est[s][n] = sum_{c < n_colours} sum_{a} v_{s,c,a}^H P_{p_n} A^{-1} v_{s,c,a}
 * for noise sets s = set0 .. set0 + n_sets - 1, a over all dof components when
 * dilute != 0, else a = 0 only.  col_dev: int32 [N] colours in [0, n_colours)
 * (all zero gives the unprobed Hutchinson estimator).  Every probe of every set
 * is queued into one batched, graph-driven solve; converged RHS retire on the
 * device and their slot is refilled from the queue.  Accumulation in FP64.
 * est_out: host complex128 [n_sets][n_p]; mean_out: host complex128 [n_p] or
 * NULL; var_out: host float64 [n_p] or NULL, the sample variance over sets
 * (denominator n_sets - 1; zero when n_sets == 1).  Synchronises. */
PT_API int pt_trace_PAinv(pt_ctx *ctx, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                   const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets,
                   int dilute, int prec, double tol, int maxit, double *est_out,
                   double *mean_out, double *var_out, pt_stats *stats);

/* Several colourings in one batched solve (Sec. 3.3 and Sec. 4.3 compare
 * colourings and reuse one colouring for many displacements): colouring i is
 * cols_dev[i * N .. (i+1) * N) with n_colours[i] colours (host array); every
 * probe of every colouring and set is queued into the same engine run, and
 * every solve is contracted with every displacement in p_list.
 *   est_out[i][s][n] (host complex128 [n_col][n_sets][n_p])
 *     = sum_{c < n_colours[i]} sum_a v_{s,c,a}^H P_{p_n} A^{-1} v_{s,c,a}
 * with v built from colouring i.  The noise of set s is the same for every
 * colouring.  Other arguments as pt_trace_PAinv.  Synchronises. */
PT_API int pt_trace_PAinv_multi(pt_ctx *ctx, const pt_op *op, int n_col, const int32_t *cols_dev,
                                const int *n_colours, int mu, const int *p_list, int n_p, int noise,
                                uint64_t seed, int set0, int n_sets, int dilute, int prec, double tol,
                                int maxit, double *est_out, pt_stats *stats);

/* Estimates at every level of a nested colouring from the solves of its
 * finest level only (the hierarchical reading of a colouring grown from k1 up
 * to k; see pt_colour_nested).  cols_dev[l * N .. (l+1) * N), l = 0 (coarsest)
 * .. n_lev - 1 (finest), must be nested: nodes with the same level-(l+1)
 * colour share their level-l colour (PT_ERR_ARG otherwise).  Only the probes
 * of the finest classes are solved; since the probes of the finer classes
 * inside a level-l class sum to its probe (Eq. (4), shared noise), the
 * level-l solution of that class is the sum of theirs, and each finest solve
 * is contracted with its ancestor's probe at every level:
 *   est_out[l][s][n] (host complex128 [n_lev][n_sets][n_p])
 *     = sum_{c_l} sum_a v_{s,c_l,a}^H P_{p_n} A^{-1} v_{s,c_l,a},
 * the pt_trace_PAinv_multi result for colouring l, at the cost of the finest
 * level's solves.  n_lev * n_p <= 32.  A temporary stream-ordered
 * allocation holds the ancestor table.  Other arguments as pt_trace_PAinv.
 * Synchronises. */
PT_API int pt_trace_PAinv_nested(pt_ctx *ctx, const pt_op *op, int n_lev, const int32_t *cols_dev,
                                 const int *n_colours, int mu, const int *p_list, int n_p, int noise,
                                 uint64_t seed, int set0, int n_sets, int dilute, int prec, double tol,
                                 int maxit, double *est_out, pt_stats *stats);

/* ---------------------------------------------------------------- deflation */

/* Deflation of given triplets (Sec. 2.4, Eq. (6)) for the displaced trace.
 * With U, V (n_ev columns each) and M = (U^H A V)^{-1} (the caller's small
 * matrix; for singular triplets, diag(1 / sigma)):
 *   Tr(P A^{-1}) = Tr(M U^H P V) + Tr(P A^{-1} (I - Q)),  Q = A V M U^H,
 * and a probe v contributes v^H P A^{-1} v - (v^H P V) M (U^H v) to the
 * second part.  This call computes the pieces that need no solve, for the
 * diluted probes of pt_trace_PAinv (same col_dev, colours, noise, seed and
 * sets; every component diluted):
 *   exact_out[n] = Tr(M U^H P_{p_n} V)                   (host complex128 [n_p])
 *   corr_out[s][n] = sum_{c,a} (v^H P_{p_n} V) M (U^H v)  (host complex128 [n_sets][n_p]),
 * so that est[s][n] - corr_out[s][n] (est from pt_trace_PAinv or
 * pt_trace_PAinv_multi) estimates the second part and exact_out + the mean
 * of that the whole trace.  U_dev, V_dev: complex128 [n_ev][N][dof] (device,
 * read; dof = 1 or 12, site-major as the user layout); M_host: complex128
 * [n_ev][n_ev] row-major (host).  1 <= n_p <= 16, 1 <= n_ev <= 4096.  The
 * per-probe and Gram dot products run on the device (temporary stream-ordered
 * allocations); the n_ev x n_ev contractions with M on the host.
 * Synchronises. */
PT_API int pt_deflation_terms(pt_ctx *ctx, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                              const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets,
                              int n_ev, const double *U_dev, const double *V_dev, const double *M_host,
                              double *corr_out, double *exact_out);

/* Eigenpairs of a small dense Hermitian matrix on the host: the Rayleigh-Ritz
 * step of pt_singular_triplets, exported for its own tests (no paper
 * counterpart; a textbook routine: Householder tridiagonalisation, a diagonal
 * phase that makes the tridiagonal real, the symmetric QR algorithm with
 * implicit Wilkinson shifts).  T_host: complex128 [m][m] row-major (host,
 * read; its Hermitian part (T + T^H) / 2 is used); w_out: float64 [m] (host),
 * every eigenvalue ascending; X_out: complex128 [n_vec][m] (host), the
 * eigenvectors of the lowest n_vec, orthonormal.  1 <= m <= 4096,
 * 0 <= n_vec <= m.  PT_ERR_NUMERIC on a non-finite entry.  No device work. */
PT_API int pt_hermitian_eig(int m, const double *T_host, int n_vec, double *w_out, double *X_out);

/* The lowest singular triplets that deflation uses (Sec. 2.4): n_ev smallest
 * singular values of A with left / right singular vectors, A V = U diag(s).
 * Block Lanczos with full reorthogonalisation on the Hermitian operator
 * H = A (the Laplacian: symmetric positive definite, so U = V and s are its
 * eigenvalues) or H = A^H A = (g5 A)^2 (Wilson-Dirac, g5-Hermitian: V are
 * eigenvectors of H, s = ||A v||, U = A V diag(1/s)), then Rayleigh-Ritz on
 * the basis.  Each candidate vector is orthogonalised twice against the basis
 * (classical Gram-Schmidt) and dropped when less than 1e-8 of its norm is
 * left, so a block at least as large as the multiplicity of the wanted values
 * resolves degenerate ones.  The operator runs in FP64 (pt_apply); the Gram
 * and combination kernels accumulate in FP64; the Rayleigh-Ritz
 * eigendecomposition (basis size, at most block * n_iter) runs on the host.
 *   start_dev: complex128 [block][N][dof] (device, read): the start block (the
 *              Laplacian uses its real part);
 *   U_dev, V_dev: complex128 [n_ev][N][dof] (device, written);
 *   s_out: float64 [n_ev] (host, written), ascending.
 * 1 <= block <= 64, n_iter >= 1, block * n_iter <= 1024, n_ev <= block * n_iter.
 * PT_ERR_NUMERIC if the Krylov space closes with fewer than n_ev vectors.
 * Temporary stream-ordered allocations: (2 block n_iter + 3 block) vectors.
 * Synchronises. */
PT_API int pt_singular_triplets(pt_ctx *ctx, const pt_op *op, int n_ev, int block, int n_iter,
                                const double *start_dev, double *U_dev, double *V_dev, double *s_out);

/* ---------------------------------------------------------------- even-odd */

/* Even-odd (red-black) preconditioning of both operators (the standard first
 * step towards the paper's production solver, Sec. 4.2; no equation of the
 * paper).  Every lattice side must be even (PT_ERR_ARG otherwise).  With the
 * even sites first, A = [[A_ee, A_eo], [A_oe, A_oo]] and A x = b becomes
 *   S x_e = b'_e,  S = A_ee - A_eo A_oo^{-1} A_oe,
 *   b'_e = b_e - A_eo A_oo^{-1} b_o,  x_o = A_oo^{-1} (b_o - A_oe x_e);
 * Laplacian (d = 8 + m2): S = d - H_eo H_oe / d, b'_e = b_e + H_eo b_o / d,
 * x_o = (b_o + H_oe x_e) / d; Wilson: S = 1 - kappa^2 D_eo D_oe,
 * b'_e = b_e + kappa D_eo b_o, x_o = b_o + kappa D_oe x_e.
 * A half field holds the sites of one parity in storage order: site i is
 * entry i >> 1 of its parity's half field.  Fields are in the user layout
 * (float64 [nrhs][sites] or complex128 [nrhs][sites][4][3], device), FP64
 * throughout; calls are enqueued on the context stream.
 *
 * pt_eo_layout (host only): site_out[h] (int32 [N/2]) = storage index of
 * entry h of the half field of `parity`; nbr_out[8 h + 2 mu + 0/1] (int32
 * [N/2][8]) = half-field index (in the other parity) of x + mu / x - mu. */
PT_API int pt_eo_layout(const int dims[4], int parity, int32_t *site_out, int32_t *nbr_out);

/* Clover Wilson operators (A_c = A_W + C, see pt_clover_blocks) enter
 * through their diagonal blocks: Aee = 1 + C on the even sites and
 * Aoo_inv = (1 + C)^{-1} on the odd ones, complex128 [N/2][12][12] by
 * half-field entry (device; pt_eo_clover_blocks makes both), or NULL for the
 * plain operators (Laplacian: must be NULL).  Then
 *   S = A_ee - kappa^2 D_eo A_oo^{-1} D_oe,  b'_e = b_e + kappa D_eo A_oo^{-1} b_o,
 *   x_o = A_oo^{-1} (b_o + kappa D_oe x_e).
 *
 * pt_eo_schur: ye = S xe for nrhs even half fields (xe, ye must not overlap;
 * temporary stream-ordered half fields). */
PT_API int pt_eo_schur(pt_ctx *ctx, const pt_op *op, const double *Aee_dev, const double *Aoo_inv_dev,
                       const double *xe_dev, double *ye_dev, int nrhs);

/* be = b'_e (even half fields) from full fields b. */
PT_API int pt_eo_prepare(pt_ctx *ctx, const pt_op *op, const double *Aoo_inv_dev, const double *b_dev,
                         double *be_dev, int nrhs);

/* x (full fields) = x_e on the even sites and x_o = A_oo^{-1}(b_o - A_oe x_e)
 * on the odd ones, from even half fields xe and full fields b (temporary
 * stream-ordered half fields). */
PT_API int pt_eo_reconstruct(pt_ctx *ctx, const pt_op *op, const double *Aoo_inv_dev, const double *xe_dev,
                             const double *b_dev, double *x_dev, int nrhs);

/* The clover diagonal blocks for the calls above, from a Wilson operator's
 * links: Aee_dev = 1 + C_ee, Aoo_inv_dev = (1 + C_oo)^{-1} (device, written;
 * temporary stream-ordered buffers; PT_ERR_NUMERIC if a block is singular).
 * Synchronises. */
PT_API int pt_eo_clover_blocks(pt_ctx *ctx, const pt_op *op, double csw, double *Aee_dev, double *Aoo_inv_dev);

/* The same three steps on the host, with the device entries' site arithmetic
 * and sequence of steps (no GPU needed): kind 0 (Laplacian, m2) or 1 (Wilson,
 * kappa, links U_host in the user layout, antip, optional clover blocks Aee,
 * Aoo_inv as above); step 0: out = S in1 (even half fields), 1: out = b'_e
 * from full fields in1, 2: out = full x from even half fields in1 and full
 * fields in2.  Host buffers. */
PT_API int pt_eo_host(int kind, const int dims[4], double m2, double kappa, const double *U_host, int antip,
                      const double *Aee, const double *Aoo_inv, int step, const double *in1, const double *in2,
                      double *out, int nrhs);

/* A x = b through the even system, for nrhs full fields (user layout,
 * device; x and b must not overlap): b'_e (pt_eo_prepare), S x_e = b'_e from
 * x_e = 0 by CG (Laplacian: S is symmetric positive definite) or BiCGStab
 * (Wilson, clover: restarted from the true residual) in FP64 until
 * ||b'_e - S x_e|| <= tol ||b'_e||, then the reconstruction.  One right-hand
 * side at a time; each dot product is summed in a fixed order and read back
 * (the building-block solver, not the batched engine).  iters_out (int32
 * [nrhs]) and relres_out (float64 [nrhs], the even system's true relative
 * residual): host, may be NULL.  PT_ERR_NOCONV if a right-hand side reaches
 * maxit first (outputs still written).  Synchronises. */
PT_API int pt_eo_solve(pt_ctx *ctx, const pt_op *op, const double *Aee_dev, const double *Aoo_inv_dev,
                       const double *b_dev, double *x_dev, int nrhs, double tol, int maxit, int *iters_out,
                       double *relres_out);

/* The same solve on the host (no GPU; the same steps, host buffers). */
PT_API int pt_eo_solve_host(int kind, const int dims[4], double m2, double kappa, const double *U_host, int antip,
                            const double *Aee, const double *Aoo_inv, const double *b, double *x, int nrhs,
                            double tol, int maxit, int *iters_out, double *relres_out);

/* Probed estimates of Tr(P_{p_n} A^{-1}) for the shifted Laplacian with the
 * solves on the even Schur complement: the same tasks, sources, contraction
 * and output as pt_trace_PAinv (est_out: host complex128 [n_sets][n_p]; the
 * colouring col_dev on the device), each task solving S x_e = b'_e by FP32 CG
 * (to delta times its starting residual) inside FP64 defect correction to
 * ||b'_e - S x_e|| <= tol ||b'_e||, then x_o = (v_o + H_oe x_e) / d where the
 * contraction reads it.  The tasks of a batch advance in lockstep (batch size
 * bounded by the memory budget and the slot cap); per-task scalars are
 * computed on the host after one reduction per step.  Every lattice side
 * even; 1 <= n_p <= 32.  stats: n_rhs, inner and outer iterations,
 * site_rhs_applies (inner iterations x N), kernel launches, largest final
 * relative residual of the even system, n_slots = batch size.  noise must be
 * PT_NOISE_Z2 (the operator is real; PT_ERR_ARG otherwise).
 * PT_ERR_NOCONV if a task reaches maxit (est_out still written).
 * Synchronises. */
PT_API int pt_trace_PAinv_eo(pt_ctx *ctx, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                             const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets, double tol,
                             int maxit, double delta, double *est_out, pt_stats *stats);

/* The same estimates on the host (no GPU; the same steps; col_host on the
 * host; all tasks in one batch). */
PT_API int pt_trace_PAinv_eo_host(const int dims[4], double m2, const int32_t *col_host, int n_colours, int mu,
                                  const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets,
                                  double tol, int maxit, double delta, double *est_out, pt_stats *stats);

/* ---------------------------------------------------------------- multigrid */

/* Two-level multigrid for the shifted Laplacian as a CG preconditioner (the
 * paper solves with an adaptive multigrid library, Sec. 4.2, and describes
 * none of its method; this is the textbook aggregation scheme).  Aggregates:
 * blocks of block^4 sites (block must divide every side); prolongator: the
 * normalised block indicators, so the Galerkin coarse operator is
 * P^T A P = A_coarse(block m2) / block; the cycle M: nu damped-Jacobi sweeps
 * (weight omega) from zero, the coarse correction (coarse CG to 1e-13), nu
 * sweeps, symmetric positive definite.  pt_mg_solve: A x = b for nrhs fields
 * (float64 [nrhs][N], device; x and b must not overlap) by M-preconditioned
 * CG from x = 0 in FP64 to ||b - A x|| <= tol ||b||, one right-hand side at
 * a time; iters_out (int32 [nrhs]) and relres_out (float64 [nrhs], the true
 * relative residual): host, may be NULL.  PT_ERR_NOCONV if a right-hand side
 * reaches maxit first.  1 <= block, 0 <= nu <= 16, 0 < omega <= 1.
 * Synchronises. */
PT_API int pt_mg_solve(pt_ctx *ctx, const pt_op *op, int block, int nu, double omega, const double *b_dev,
                       double *x_dev, int nrhs, double tol, int maxit, int *iters_out, double *relres_out);

/* The same solve on the host, and one application out = M r of the cycle
 * (host buffers; the same site arithmetic and steps; no GPU). */
PT_API int pt_mg_solve_host(const int dims[4], double m2, int block, int nu, double omega, const double *b,
                            double *x, int nrhs, double tol, int maxit, int *iters_out, double *relres_out);
PT_API int pt_mg_cycle_host(const int dims[4], double m2, int block, int nu, double omega, const double *r,
                            double *out);

/* Two-level adaptive aggregation multigrid for the Wilson-Dirac operator as a
 * right preconditioner of FGMRES (the textbook construction; the paper's
 * adaptive multigrid library is not described, Sec. 4.2): aggregates are
 * blocks of block^4 sites split by chirality; nv near-null vectors are
 * counter-based random vectors (seed) relaxed by `sweeps` damped Richardson
 * sweeps (weight omega) on A v = 0, restricted to each aggregate and
 * orthonormalised; A_c = P^H A P is a nine-point block stencil on the coarse
 * lattice; the cycle is nu Richardson sweeps, the coarse correction (A_c by
 * BiCGStab to 1e-10) and nu sweeps; FGMRES(restart) from x = 0 to
 * ||b - A x|| <= tol ||b||.  b_dev, x_dev: complex128 [nrhs][N][4][3]
 * (device); iters_out (int32 [nrhs]) and relres_out (float64 [nrhs], true
 * relative residual): host, may be NULL.  1 <= nv <= 8, 6 block^4 >= nv,
 * 1 <= restart <= 64, 0 <= nu <= 16.  PT_ERR_NOCONV if a right-hand side
 * reaches maxit first.  csw != 0 makes the operator the clover one, A_W + C
 * (pt_clover_blocks; a temporary stream-ordered copy of the blocks).
 * Synchronises. */
PT_API int pt_wmg_solve(pt_ctx *ctx, const pt_op *op, double csw, int block, int nv, int sweeps, int nu,
                        double omega, int restart, uint64_t seed, const double *b_dev, double *x_dev, int nrhs,
                        double tol, int maxit, int *iters_out, double *relres_out);

/* The same solve on the host (links U_host in the user layout; no GPU), and
 * the setup alone: P_out complex128 [Nc][2][nv][block^4][6] (coarse site,
 * chirality half, vector, site in the block, spin-colour component in the
 * half) and Ac_out complex128 [Nc][9][2 nv][2 nv] (stencil slot 0 = self,
 * 1 + 2 mu = +mu, 2 + 2 mu = -mu). */
PT_API int pt_wmg_solve_host(const int dims[4], const double *U_host, double kappa, double csw, int antip, int block,
                             int nv, int sweeps, int nu, double omega, int restart, uint64_t seed, const double *b,
                             double *x, int nrhs, double tol, int maxit, int *iters_out, double *relres_out);
PT_API int pt_wmg_setup_host(const int dims[4], const double *U_host, double kappa, double csw, int antip, int block,
                             int nv, int sweeps, double omega, uint64_t seed, double *P_out, double *Ac_out);

/* ---------------------------------------------------------------- clover */

/* Clover (Sheikholeslami-Wohlert) site blocks of the Wilson-Dirac operator
 * (Sec. 4.2 names a clover Wilson operator and leaves its definition to the
 * literature; the textbook form with this library's gamma basis and hopping
 * sign):
 *   C(x) = -kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
 *   sigma_{mu nu} = (i/2)[g_mu, g_nu],  F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^H)/(8 i),
 * Q_{mu nu}(x) the four plaquettes of the (mu, nu) plane at x, so that the
 * clover operator is A_c = A_W + C.  Blocks: complex128 [N][12][12],
 * row-major, component = 3 spin + colour.  The per-site arithmetic is shared
 * by the device kernels and the host-only entries (which need no GPU).
 *
 * pt_clover_blocks_host: from links in the user layout (host, complex128
 * [N][4][3][3]); blocks_out on the host.  pt_clover_blocks: from the links of
 * a Wilson operator; blocks_dev on the device (enqueued on the stream). */
PT_API int pt_clover_blocks_host(const int dims[4], const double *U_host, double kappa, double csw,
                                 double *blocks_out);
PT_API int pt_clover_blocks(pt_ctx *ctx, const pt_op *op, double csw, double *blocks_dev);

/* The clover Wilson operator A_c = A_W + C (C as in pt_clover_blocks, Sec. 4.2)
 * in the batched engine: pt_op_set_clover(op, csw) gives the Wilson operator
 * op the clover term with coefficient csw (csw = 0 removes it).  It computes
 * the site blocks 1 + C(x) and their inverses (FP64, on the device), checks
 * that each is two Hermitian 6 x 6 chiral blocks, and keeps them packed with
 * the operator (FP64, plus an FP32 copy for the inner solves): about
 * 1.7 KB + 0.6 KB per even-odd site pair.  From then on pt_apply applies
 * A_W + C (the term added in FP64), and pt_solve, pt_trace_PAinv and
 * pt_trace_multi solve with A_c on the even Schur complement
 * S = A_ee - kappa^2 D_eo A_oo^{-1} D_oe (b'_e = b_e + kappa D_eo A_oo^{-1} b_o,
 * x_o = A_oo^{-1} (b_o + kappa D_oe x_e)) with the stopping test of the full
 * system; the engine's even-odd mode is then always on and the link-sharing
 * groups (rhs_block 8) are not used.  Errors: PT_ERR_ARG if op is not a
 * Wilson operator or a side of the lattice is odd (the engine also refuses
 * pt_grad on a clover operator); PT_ERR_NUMERIC if a block 1 + C(x) is
 * singular or not of the chiral Hermitian form (the operator keeps its
 * previous term); PT_ERR_OOM.  Synchronises; temporary device buffers of
 * 2 x 2.3 KB per site while it runs.  The building-block entry points
 * (pt_eo_*, pt_wmg_solve) take their clover blocks or c_sw explicitly and do
 * not use the operator's term. */
PT_API int pt_op_set_clover(pt_op *op, double csw);

/* y[r][x] = beta y[r][x] + B(x) x[r][x] for nrhs spinor fields (user layout,
 * device; x and y must not overlap) and blocks B [N][12][12] (device).  With
 * beta = 1 and y = A_W x (pt_apply) this is the clover operator. */
PT_API int pt_site_blocks_apply(pt_ctx *ctx, int N, const double *blocks_dev, const double *x_dev, double beta,
                                double *y_dev, int nrhs);

/* inv = (shift 1 + B(x))^{-1} per site by Gauss-Jordan elimination with
 * partial pivoting (shift = 1 gives the clover diagonal block A_xx);
 * PT_ERR_NUMERIC if a block is singular.  _host: n blocks on the host; the
 * device form synchronises the stream. */
PT_API int pt_site_blocks_invert_host(int n, const double *blocks, double shift, double *inv_out);
PT_API int pt_site_blocks_invert(pt_ctx *ctx, int N, const double *blocks_dev, double shift, double *inv_dev);

/* ---------------------------------------------------------------- gradient */

/* Adjoint gradient of the probed estimate T = sum_s est[s] for one
 * displacement p (not in the paper): with x = A^{-1} v, y = A^{-+} P^T v,
 *   dT/dtheta = - sum_v y^H (dA/dtheta) x.
 * Laplacian: *dparam_out = dT/dm2 (complex128, host).  Wilson: dT/dkappa, and,
 * if G_dev / Gbar_dev are not NULL, the link derivatives (user link layout,
 * device, overwritten)
 *   G_mu(x)_ab    = dT/dU_mu(x)_ab,   Gbar_mu(x)_ab = dT/d conj(U_mu(x)_ab)
 * (entries of U treated as free complex numbers).  Forward and adjoint solves
 * are recomputed (no Krylov history is stored); the adjoint solve uses
 * A^{-+} = g5 A^{-1} g5.  est_out: host complex128 [n_sets] or NULL.
 * Synchronises. */
PT_API int pt_grad(pt_ctx *ctx, const pt_op *op, const int32_t *col_dev, int n_colours, int mu, int p,
            int noise, uint64_t seed, int set0, int n_sets, int dilute, int prec, double tol,
            int maxit, double *est_out, double *dparam_out, double *G_dev, double *Gbar_dev,
            pt_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* PTRACE_H */
