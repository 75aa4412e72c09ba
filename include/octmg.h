/*
 * octmg.h -- C ABI of the GB300 octree-block multigrid library (libocmg.so).
 *
 * The method is the matrix-free multigrid of arXiv 2403.08063 ("Towards Code Generation for Octree-Based
 * Multigrid Solvers"): a forest of octree blocks over the unit cube (Sec. 2), every block holding n^3
 * cell-centred unknowns plus one ghost layer (Sec. 3.3), with same-level, coarse-to-fine (quadratic, Sec. 3.3.2)
 * and fine-to-coarse (linear, Sec. 3.3.1) ghost exchange, solving -div(k grad u) = f with Dirichlet data
 * (Sec. 5, Eq. 1-2) by V-cycles whose coarse levels halve every block down to 4^3 cells (Sec. 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Field layout ("user layout"): leaf-major in the order of mg_config.leaves; each leaf holds its n^3 interior
 *    cells with x fastest, i.e. element [leaf * n^3 + (z * n + y) * n + x].  FP64.
 *  - Pointers named *_dev are CUDA device pointers, caller-owned; pointers named *_host are host pointers.
 *    Device work is ordered on mg_config.stream; a call returns after its work is enqueued unless it returns a
 *    host-visible result (residual norms, cycle counts), in which case it synchronises that stream.
 *  - The library never keeps a caller pointer beyond the call.  mg_set_rhs copies f and k into the forest.
 *  - Errors: every call returns mg_status; nothing is thrown across the ABI and no error traps the GPU.
 *    mg_last_error() returns a thread-local description of the last failure.  CUDA errors map to MG_ERR_CUDA.
 *  - Thread safety: a forest may be used by one host thread at a time.
 */
#ifndef OCTMG_H
#define OCTMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_forest mg_forest; /* opaque, library-owned */

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum value */
    MG_ERR_UNBALANCED = 2,    /* leaves do not tile the domain, overlap, or violate 2:1 face balance (Sec. 2) */
    MG_ERR_BLOCK_SIZE = 3,    /* n not a power of two >= 4 (C2F needs 3 cells per axis, Sec. 3.3.2) */
    MG_ERR_OOM = 4,           /* device or host allocation failed */
    MG_ERR_CUDA = 5,          /* a CUDA call failed */
    MG_ERR_NOT_CONVERGED = 6, /* residual did not reach rtol within max_cycles, or became non-finite */
    MG_ERR_TIMEOUT = 7,       /* a bounded device wait gave up (staged smoother copies, persistent tail barrier) */
    MG_ERR_NONFINITE = 8,     /* NaN/Inf in an input field, or k <= 0 */
    MG_ERR_STATE = 9          /* call out of order (e.g. solve before mg_set_rhs) */
} mg_status;

typedef struct {
    int32_t roots;            /* R: root blocks per axis; the roots are R^3 cubes of edge 1/R over [0,1]^3 (Sec. 2) */
    int32_t n;                /* cells per block edge on the finest level; power of two, >= 4 */
    int32_t n_leaves;
    const int32_t *leaves;    /* host, 5 * n_leaves int32: (problem, level, i, j, k), problem in 0..n_problems-1.
                                 Leaf (level, i, j, k) covers [i, i+1] x [j, j+1] x [k, k+1] / (R 2^level) of its
                                 problem's unit cube; every problem's leaves must tile its cube, 2:1 face balanced. */
    int32_t coeff;            /* 0: -Laplace(u) = f;  1: -div(k grad u) = f with per-cell k > 0 */
    int32_t interface_flux;   /* 1 (default): conservative coarse-fine faces (the coarse flux is the sum of the four
                                 fine sub-face fluxes); 0: the paper's ghost-only scheme (coarse ghost = F2C mean) */
    int32_t precision;        /* 0: FP64 V-cycles; 1: FP32 V-cycles inside FP64 defect correction */
    int32_t nu1, nu2;         /* pre/post red-black Gauss-Seidel iterations (2, 2) */
    int32_t max_coarse;       /* octets are merged below 4^3 blocks until the coarsest level has at most this many
                                 unknowns (default 512 when <= 0); that level is solved by a dense FP64 inverse */
    int32_t inner_cycles;     /* precision == 1: FP32 V-cycles per FP64 defect-correction step (default 1 when <= 0;
                                 FP32 resolves about 6 digits per step, so up to ~5 cycles still pay) */
    int32_t n_problems;       /* independent problems sharing R and n, solved together (default 1 when <= 0) */
    void *stream;             /* cudaStream_t, or NULL for the legacy default stream */
    /* The paper's own cycle and interpolation variants (Sec. 5, Table err_analysis); zero keeps the defaults. */
    int32_t c2f_variant;      /* coarse-to-fine ghosts: 0 quadratic (Sec. 3.3.2), 1 first order, 2 constant (the
                                 lower orders of Table err_analysis, not described in the paper: readings) */
    int32_t smoother;         /* 0 red-black Gauss-Seidel; 1 damped Jacobi, one sweep per smoothing step (FP64) */
    double omega;             /* Jacobi damping (0.8 when <= 0) */
    int32_t coarse_iters;     /* 0: dense direct coarsest solve; > 0: that many damped Jacobi sweeps (FP64) */
    int32_t coarse_coef;      /* coeff == 1, coarse levels: 0 rediscretised from k, the mean of the 8 children's
                                 (default); 1 every coarse face takes the mean of the 2 x 2 finer face coefficients
                                 it covers (an operator-aware coarsening not in the paper; far fewer V-cycles for
                                 rough k).  The finest level's coefficients are the harmonic means either way. */
    int32_t prolongation;     /* 0 face-neighbour linear (each fine cell from its coarse cell and the three face
                                 neighbours towards it; default); 1 trilinear (8 coarse cells), which reads the coarse
                                 correction's edge and corner ghosts: copies from a same-level block across the edge
                                 or corner, else linear extrapolation from the neighbouring face (edge) ghosts (the
                                 diagonal ghosts of the paper's future work, Sec. 8).  With 1 the persistent tail is
                                 off and mg_adjoint_solve returns MG_ERR_INVALID_ARG; mg_exchange_level also fills
                                 the edge and corner ghosts. */
} mg_config;

/* Build the forest: validate the leaves, build neighbour and segment tables for every multigrid level, allocate
 * device pools.  For coeff == 0 the coarsest-level inverse is assembled here; for coeff == 1 in mg_set_rhs.
 * Errors: MG_ERR_INVALID_ARG, MG_ERR_BLOCK_SIZE, MG_ERR_UNBALANCED, MG_ERR_OOM, MG_ERR_CUDA.  On error *out = NULL. */
mg_status mg_forest_create(const mg_config *cfg, mg_forest **out);

/* Free every device and host buffer of the forest (synchronises its stream).  NULL is a no-op.  No counterpart in
 * the paper, whose generated code keeps its blocks for the program's lifetime (Sec. 4); the lifetime call belongs to
 * this library's C ABI. */
void mg_forest_destroy(mg_forest *forest);

/* Number of multigrid levels, and (optionally) per level the block count and block edge (host arrays of
 * n_levels entries, either may be NULL).  Level 0 is the finest; each coarser level halves every block's edge
 * (block-local coarsening, Sec. 5) down to 4^3, then merges complete sibling octets while the coarsest level has
 * more than max_coarse unknowns (this library's addition for a dense coarsest solve). */
mg_status mg_forest_levels(const mg_forest *forest, int32_t *n_levels, int32_t *nb_per_level, int32_t *n_per_level);

/* Block keys (level, i, j, k) of multigrid level `level`, in the level's block order (keys_host: 4 * nb int32);
 * (level, i, j, k) names the octree block of edge 1 / (R 2^level) at (i, j, k) (Sec. 2). */
mg_status mg_level_keys(const mg_forest *forest, int32_t level, int32_t *keys_host);

/* Copy the right-hand side f of -div(k grad u) = f (Sec. 5, Eq. 1; a per-cell k is the variable coefficient that
 * Sec. 8 names as future work) and, for coeff == 1, the coefficient k into the forest; for coeff == 1 also build
 * the face coefficients (harmonic means of the two cells' k), the coefficient pyramid (k of a coarse cell = mean
 * of its 8 children) and the coarsest-level inverse.
 * f_dev: n_leaves * n^3 doubles; k_dev: same size, every entry finite and > 0, or NULL when coeff == 0.
 * Errors: MG_ERR_INVALID_ARG, MG_ERR_NONFINITE, MG_ERR_CUDA. */
mg_status mg_set_rhs(mg_forest *forest, const double *f_dev, const double *k_dev);

/* Inhomogeneous Dirichlet data g (Sec. 5, Eq. 2) for the finest level: g_dev (device, FP64) holds, per leaf in
 * leaf order, its 6 faces (face = 2 axis + side, side 1 = the upper face) of n^2 values each, index i2 * n + i1 with
 * (i1, i2) the interior coordinates along the two other axes in increasing axis order; only faces on the domain
 * boundary are read.  The boundary ghost becomes 2 g - u (the value g at the face centre).  NULL restores g = 0.
 * Coarse levels (corrections) keep g = 0.  Relative residuals are then taken against the residual of u = 0.  Used
 * by FP64 cycles and by the FP64 residual of FP32-in-FP64 solves; the adjoint rejects a forest with g set. */
mg_status mg_set_boundary(mg_forest *forest, const double *g_dev);

/* Run exactly ncycles V(nu1, nu2) cycles (Sec. 5: smoothing with the ghosts refreshed before every half-sweep
 * (Sec. 3), residual, 8:1 restriction, coarser levels, prolongation and correction) on u_dev (initial guess on
 * entry, iterate on exit; FP64 cycles, or FP32 cycles inside FP64 defect correction when precision == 1).  If rel_res_out is not NULL it receives, per problem
 * (n_problems doubles), ||f - A u|| / ||f|| after the last cycle (volume-weighted L2 norm sqrt(sum h^3 r^2) over that
 * problem's cells).  Requires mg_set_rhs. */
mg_status mg_vcycle(mg_forest *forest, double *u_dev, int32_t ncycles, double *rel_res_out);

/* Cycle from the initial guess in u_dev until every problem has ||f - A u|| / ||f|| <= rtol (the relative L2
 * residual criterion of Sec. 5, volume-weighted), or max_cycles cycles ran.  cycles_out / rel_res_out (host arrays of n_problems entries, may be NULL) receive per problem the number of
 * cycles after which it first met rtol (or the total) and its final relative residual.  All problems keep cycling
 * until the last one converges.  Returns MG_ERR_NOT_CONVERGED (u_dev still holds the last iterate) when a problem
 * does not reach rtol. */
mg_status mg_solve(mg_forest *forest, double *u_dev, double rtol, int32_t max_cycles, int32_t *cycles_out,
                   double *rel_res_out);

/* mg_set_rhs + mg_solve from host buffers (user layout, FP64, n_leaves * n^3 each): f_host, k_host (NULL when
 * coeff == 0), u0_host the initial guess (NULL: zero), u_host receives the solution (may be the same buffer as
 * u0_host).  The library copies into device staging buffers of its own (allocated at the first call, kept by the
 * forest): k first on the forest's stream, where its set-up (coefficient pyramid, coarsest inverse) starts while f
 * and the initial guess cross on a second stream; the solve then runs as mg_solve and u is copied back.  Page-locked
 * host buffers let the copies run at full bandwidth and overlap; pageable ones work too.  Returns when u_host holds
 * the result (or on error).  Errors as mg_set_rhs and mg_solve; MG_ERR_STATE for a forest of a batch. */
mg_status mg_solve_host(mg_forest *forest, const double *f_host, const double *k_host, const double *u0_host,
                        double *u_host, double rtol, int32_t max_cycles, int32_t *cycles_out, double *rel_res_out);

/* Adjoint of the converged solve (this library's extension; the paper has no adjoint) for
 * L = 1/2 sum_i (u_i - u_t,i)^2: given u_dev (the forward solution) and
 * dLdu_dev = u - u_t, solve A^T lambda = dL/du by defect correction with the transposed V-cycle, write lambda
 * (= dL/df) to lambda_dev and, when dLdk_dev is not NULL and coeff == 1, dL/dk = -lambda^T (dA/dk) u.
 * All arrays n_leaves * n^3 doubles on the device.  With several problems, rtol applies to the norm over all of
 * them.  Returns MG_ERR_NOT_CONVERGED if rtol is not reached. */
mg_status mg_adjoint_solve(mg_forest *forest, const double *u_dev, const double *dLdu_dev, double *lambda_dev,
                           double *dLdk_dev, double rtol, int32_t max_cycles);

/* The finest-level operator of Sec. 5, Eq. 1-2: Au_dev = A u_dev (ghosts filled by the full exchange of Sec. 3,
 * homogeneous Dirichlet data), and its transpose ATy_dev = A^T y_dev.  Requires mg_set_rhs when coeff == 1. */
mg_status mg_apply(mg_forest *forest, const double *u_dev, double *Au_dev);
mg_status mg_apply_transpose(mg_forest *forest, const double *y_dev, double *ATy_dev);

/* Debug view of one exchange (Sec. 3.1 same level, Sec. 3.3.2 coarse to fine, Sec. 3.3.1 fine to coarse, and the
 * Dirichlet reflection at the domain boundary): copy u_dev (user layout of level `level`, nb_level * n_level^3
 * doubles) into the level's FP64 pool, run that level's ghost exchange, and copy the whole padded pool (nb_level * (n_level+2)^3
 * doubles, block-major, x fastest) to padded_dev. */
mg_status mg_exchange_level(mg_forest *forest, int32_t level, const double *u_dev, double *padded_dev);

/* mg_exchange_level without device allocation.  The paper has no counterpart: this serves callers that cannot let
 * a library call cudaMalloc when they need the exchange -- applications whose device memory is entirely owned by a
 * caching allocator or reserved at start-up, and loops with a latency budget that must not enter CUDA's device
 * allocator.  Same arguments and result as mg_exchange_level, but the level's padded scratch pool is a static
 * device array of 524,288 doubles (4 MiB) inside the library, which every GPU that loads the library holds until
 * the process exits; a level whose pool (nb * (n+2)^3 rounded up to 32 doubles per block) is larger is rejected
 * with MG_ERR_INVALID_ARG and a message.  Nothing else is allocated either: on a variable-k forest with FP32
 * cycles (precision 1) and conservative interfaces, the FP64 face coefficients that the fine-to-coarse ghosts
 * need are created by the first mg_exchange_level, mg_apply or mg_adjoint_solve call; before that, a level with
 * fine-to-coarse ghosts returns MG_ERR_STATE.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any CUDA stream capture starts in the process.
 * All calls share the array and it keeps the last call's contents (each
 * call clears the part it uses): calls whose work overlaps on the GPU (other streams, other threads, other
 * forests) race on it.  The call enqueues its work on the forest's stream and synchronises that stream before
 * returning. */
mg_status mg_exchange_level_noalloc(mg_forest *forest, int32_t level, const double *u_dev, double *padded_dev);

/* Kernel accounting (no counterpart in the paper).  Launch counters per kernel family always run; mg_profile(forest, 1) clears them and starts
 * recording a CUDA-event pair on the forest's stream around every family's launches, mg_profile(forest, 0) stops.
 * mg_profile_read synchronises the stream and, for up to max_families families, writes the family name (32 bytes
 * each, NUL-terminated) into names, the summed event time in milliseconds into ms and the launch count into
 * launches (each output may be NULL); *n_families receives the number of families. */
mg_status mg_profile(mg_forest *forest, int32_t enable);
mg_status mg_profile_read(mg_forest *forest, int32_t max_families, char *names, double *ms, int64_t *launches,
                          int32_t *n_families);

/* Launch shape of the FP32 smoother on one level (precision 1, block edges 4..128), five int32 {kind, p1..p4}:
 *   {1, zc, threads, 0, 0}: one thread per zc cells of a z-column (zc 1, 2 or 4), CTAs of 128, 256 or 512 threads;
 *   {2, TY, TZ, D, R}:      edges 32..128: a CTA per TY rows x TZ planes of a block, the other colour's planes
 *                           staged in shared memory by bulk copies D planes ahead, R rows per thread (with
 *                           variable k 1/k, on face-averaged coarse levels the three face arrays, of both colours,
 *                           are staged too).
 * mg_smoother_shapes lists the shapes offered for a level (5 int32 each, up to max_shapes into shapes, which may
 * be NULL; *n_shapes receives the count).  The first mg_set_rhs of a forest picks each level's shape by timing
 * every offered shape on the level's own FP32 pools (levels under 2^18 cells take {1, 1, 256, 0, 0}); the choice
 * is cached for the process per (device, coefficient mode, n, block count).  mg_set_smoother_shape overrides it.
 * A shape only changes which thread updates a cell, so every shape gives bit-identical results.
 * get: all zeros for a level that uses the generic smoother (FP64 solves, n > 128) or is not tuned yet.
 * set: MG_ERR_INVALID_ARG for a bad level, a shape not offered, or a level without the specialised smoother.
 * No counterpart in the paper, whose kernels are generated per block size (Sec. 4). */
mg_status mg_smoother_shapes(const mg_forest *forest, int32_t level, int32_t max_shapes, int32_t *shapes,
                             int32_t *n_shapes);
mg_status mg_get_smoother_shape(const mg_forest *forest, int32_t level, int32_t *shape);
mg_status mg_set_smoother_shape(mg_forest *forest, int32_t level, const int32_t *shape);

/* Bulk-copy plan of the staged FP32 smoother (k_smooth32t), computed on the host by the same code the kernel's
 * producer thread runs; no GPU is needed.  No counterpart in the paper: it lets a test check every shared-memory copy
 * of the kernel against the rules of cp.async.bulk without running it.  For block edge 2^lg (lg 5..7), coefficient
 * mode coeff (0 constant, 1 variable k with 1/k staged, 2 stored halved face coefficients of a face-averaged coarse
 * level, ax, ay, az staged) and half-sweep colour `colour`, *n_shapes receives the number of staged
 * shapes ({2, TY, TZ, D, R}) offered; for the one with index shape_index (none: *n_records = 0) shape receives it
 * (5 int32, may be NULL), *smem_bytes the dynamic shared memory a CTA is launched with and *block_bytes the block
 * stride of an FP32 pool (either may be NULL), and records (max_records x 10 int64, may be NULL) every mbarrier arm and
 * bulk copy that the CTAs of one block issue, in issue order per CTA:
 *   {tile (tz * n / TY + ty), kind (0 arm, 1 copy), barrier (0 first planes, 1 + g % (D + 1) group g),
 *    group g (-1: first planes), dst (bytes from the start of dynamic shared memory; -1 for an arm),
 *    array (0 other-half u, 1 other-half kappa or ax, 2 own-half f, 3 own-half kappa or ax, 4 / 5 other-half
 *    ay / az, 6 / 7 own-half ay / az; -1), src (bytes from the start of
 *    the block in the pool; -1), bytes (armed or copied), lead (floats from the copy's start to the wanted plane
 *    segment; -1), len (floats of the wanted segment; -1)}.
 * *n_records receives the total (records beyond max_records are counted, not written).  MG_ERR_INVALID_ARG for a
 * bad lg, coeff, colour or a null count pointer. */
mg_status mg_staged_copy_plan(int32_t lg, int32_t coeff, int32_t colour, int32_t shape_index, int32_t *shape,
                              int32_t *n_shapes, int64_t *smem_bytes, int64_t *block_bytes, int64_t max_records,
                              int64_t *records, int64_t *n_records);

/* Bulk-copy plan of the staged FP32 residual + restriction (k_residual_restrict32t, fine block edges 64 and 128),
 * computed on the host by the same code the kernel's producer thread runs; no GPU is needed.  No counterpart in the
 * paper: it lets a test check every shared-memory copy against the rules of cp.async.bulk without running the kernel.
 * For fine block edge 2^lg (lg 6 or 7) and coefficient mode coeff (0 constant, 1 variable k, 2 stored halved face
 * coefficients), shape (3 int32, in and out) = {TY, TZ, D}: fine rows and planes per CTA and planes staged beyond the
 * four a coarse plane reads; {0, ...} on input selects the tile the library launches, written back.  *smem_bytes
 * receives the dynamic shared memory of a CTA and *block_bytes the block stride of an FP32 pool (either may be NULL);
 * records (max_records x 11 int64, may be NULL) every mbarrier arm and bulk copy the CTAs of one block issue, in issue
 * order per CTA:
 *   {tile (tz * n / TY + ty), kind (0 arm, 1 copy), ring slot, plane q (padded plane z0 + q), dst (bytes from the
 *    start of dynamic shared memory; -1), array (0 u, then kappa (coeff 1) or ax, ay, az (coeff 2), then f; -1),
 *    half (-1), src (bytes from the start of the block in the pool; -1), bytes (armed or copied), lead (floats from
 *    the copy's start to the wanted segment; -1), len (floats of the wanted segment; -1)}.
 * *n_records receives the total (records beyond max_records are counted, not written).  MG_ERR_INVALID_ARG for a bad
 * lg, coeff or tile, or a null shape or count pointer. */
mg_status mg_restrict_copy_plan(int32_t lg, int32_t coeff, int32_t *shape, int64_t *smem_bytes, int64_t *block_bytes,
                                int64_t max_records, int64_t *records, int64_t *n_records);

/* Persistent tail of the FP32 V-cycle (precision 1): from level `level` down to the coarsest and back, every step
 * (half-sweeps, exchanges, restriction, prolongation, coarsest solve) runs inside one cooperative kernel launch
 * whose CTAs stay resident and meet at grid barriers, instead of one launch per step.  Results are bit-identical
 * to the launched V-cycle.  The first mg_set_rhs times V-cycles without the tail and with it from every level
 * whose own and deeper levels have at most 2^20 cells, and keeps the fastest.  get: -1 when off.  set: -1: off;
 * MG_ERR_INVALID_ARG for a level with a deeper block edge outside 4..128 or a forest without FP32 cycles.  A grid
 * barrier that waits too long makes the solve return MG_ERR_TIMEOUT.  No counterpart in the paper, whose cycle
 * runs level by level with MPI exchanges (Sec. 4). */
mg_status mg_get_tail(const mg_forest *forest, int32_t *level);
mg_status mg_set_tail(mg_forest *forest, int32_t level);

/* Self-test (no counterpart in the paper) of the bounded waits that keep a kernel from hanging when an expected event never comes: launches one
 * CTA on the forest's stream that waits for something nothing provides, which = 0 an mbarrier phase (the wait of the
 * staged smoother's shared-memory copies, bounded by 2^14 probes), which = 1 a grid barrier expecting one CTA more
 * than the grid has (the persistent tail's, bounded by 2^30 SM clock cycles), and reads the error word.  Expected
 * result: MG_ERR_TIMEOUT after at most about a second, with the context still usable; MG_ERR_INVALID_ARG for
 * another `which`.  Synchronises the stream. */
mg_status mg_selftest_waits(mg_forest *forest, int32_t which);

/* Measured FMA throughput of the current device (TFLOP/s, 2 flop per FMA): eight independent FMA chains per thread on
 * 8 CTAs of 256 threads per SM, one timed launch after a warm-up, on the legacy default stream; synchronises the
 * device, so call it while nothing else is queued.  FP64 (about 0.06 s) and scalar FP32 (about 0.03 s); either output
 * may be NULL, not both (MG_ERR_INVALID_ARG); MG_ERR_CUDA without a device.  The roof of the kernels bound by
 * arithmetic rather than memory (the FP64 outer residual); no counterpart in the paper. */
mg_status mg_alu_peaks(double *fp64_tflops, double *fp32_tflops);

/* ---------------------------------------------------------------------------------------------------------------
 * Batches: many independent problems with different block sizes (uneven octree forests), solved together.
 * Every problem is its own forest over [0,1]^3 with cfg->roots root blocks per axis; its leaves are the rows of
 * cfg->leaves whose problem index is p.  problem_n (host, n_problems entries, may be NULL) gives each problem's
 * block size (NULL: cfg->n for all).  Field layout: the leaves in the order of cfg->leaves, each holding its
 * problem's n_p^3 cells, x fastest.  Problems with the same n share one multi-problem forest; all run on an
 * internal stream ordered after cfg->stream on entry and before it on exit.  Solves use FP32 cycles inside FP64
 * defect correction (cfg->precision must be 1); each defect-correction step of every group is captured once in a
 * CUDA graph and replayed.  The paper solves one forest at a time (Sec. 5); batching is this library's extension.
 * --------------------------------------------------------------------------------------------------------------- */
typedef struct mg_batch mg_batch;

mg_status mg_batch_create(const mg_config *cfg, const int32_t *problem_n, mg_batch **out);
void mg_batch_destroy(mg_batch *batch);
/* f_dev, k_dev: device arrays of the batch layout (total cells doubles); k_dev NULL when cfg->coeff == 0. */
mg_status mg_batch_set_rhs(mg_batch *batch, const double *f_dev, const double *k_dev);
/* Cycle from the initial guess in u_dev (batch layout) until every problem has ||f - A u|| / ||f|| <= rtol.
 * cycles_out / rel_res_out: host arrays of n_problems entries (may be NULL), as in mg_solve. */
mg_status mg_batch_solve(mg_batch *batch, double *u_dev, double rtol, int32_t max_cycles, int32_t *cycles_out,
                         double *rel_res_out);
/* Number of block-size groups, total cells, and per group its block size and problem count (arrays may be NULL). */
mg_status mg_batch_info(const mg_batch *batch, int32_t *n_groups, int64_t *total_cells, int32_t *group_n,
                        int32_t *group_problems);
/* Kernel accounting of every group (mg_profile); while enabled, solves launch kernels without graphs. */
mg_status mg_batch_profile(mg_batch *batch, int32_t enable);
/* The multi-problem forest of group g (owned by the batch), e.g. for mg_profile_read; NULL if out of range. */
mg_forest *mg_batch_group(mg_batch *batch, int32_t g);
/* How the coarse levels of the batch's FP32 V-cycles run (the batching extension; the paper launches one forest's
 * cycle level by level, Sec. 4):
 *   0  every level of every group as separate kernel launches (each group on its own stream);
 *   1  each group's levels from its tuned tail level down (and back up) in one persistent cooperative launch of its
 *      own, concurrently with the other groups' launches;
 *   2  one joint persistent cooperative launch per V-cycle running the tails of all groups: each group first runs
 *      its levels above the tail on its own stream, then every group waits for the joint tail, then each runs its
 *      levels back up.  Between two grid barriers the joint tail runs one phase of every group.
 * mg_batch_set_rhs picks the fastest of the three on first use (two timed defect-correction steps of all groups
 * each; a persistent mode when it is within 1 % of the fastest); mg_batch_set_tail_mode overrides it (MG_ERR_STATE before mg_batch_set_rhs, MG_ERR_INVALID_ARG for another
 * mode).  All three give bit-identical iterates.  A grid barrier of the persistent launches that waits longer than
 * about half a second makes the next call return MG_ERR_TIMEOUT. */
mg_status mg_batch_set_tail_mode(mg_batch *batch, int32_t mode);
mg_status mg_batch_get_tail_mode(const mg_batch *batch, int32_t *mode);

/* Thread-local description of the last error (empty string if none); the pointer stays valid until the next failing
 * call on the same thread.  No counterpart in the paper: error reporting of this library's C ABI. */
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OCTMG_H */
