/*
 * symhss.h -- C ABI of the B300 (sm_103a) symmetric HSS direct solver for 2-D
 * Helmholtz transmission scattering (symmetric Muller-like Nystrom system).
 *
 * Problem (Sec. 2): find the boundary flux q and trace u of the field scattered
 * by a closed curve Gamma with wavenumber k0 / material constant eps0 outside
 * and k1 / eps1 inside, for an incident plane wave.  The discrete system is the
 * row-scaled symmetric Muller-like system (Eq. 15) on an equispaced-parameter
 * trapezoidal Nystrom rule with a one-point corrected diagonal (Sec. 3.1).  It is
 * compressed by the proxy method with one column interpolative decomposition per
 * box and component, reused as the row basis because the matrix is complex
 * symmetric (Sec. 4.1, Eq. low-rank_R), then factorised and solved by the
 * multilevel compressed-equation (Martinsson-Rokhlin / HSS-ULV) scheme (Sec. 4.2).
 * SYMHSS_NONSYM selects the non-symmetric baseline instead: the unscaled system of
 * Sec. 6 (naive Muller-like) with separate row and column IDs (4 IDs per box).
 *
 * Conventions
 *   - Complex numbers are complex128: two doubles (re, im), interleaved.
 *   - Unknown / equation ordering at the boundary is [q_1..q_N, u_1..u_N] and
 *     [eq1_1..eq1_N, eq2_1..eq2_N] (Eq. 15).
 *   - Every call returns an int status: SYMHSS_OK (0) or a negative error code.
 *     No call aborts the process, traps on the device or prints.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that must read results back to the host synchronise that stream.
 *   - All device memory the handle needs is allocated and owned by the handle and
 *     released by symhss_destroy.  Caller buffers are never freed by the library.
 */
#ifndef SYMHSS_H
#define SYMHSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SYMHSS_OK                  0
#define SYMHSS_ERR_INVALID        -1  /* bad size, pointer, parameter, NaN/Inf input */
#define SYMHSS_ERR_NOMEM          -2  /* device or pinned host allocation failed */
#define SYMHSS_ERR_CUDA           -3  /* a CUDA runtime call or launch failed */
#define SYMHSS_ERR_RANK_OVERFLOW  -4  /* an ID rank exceeded the preallocated capacity */
#define SYMHSS_ERR_SINGULAR       -5  /* an exactly singular pivot in a block LU */
#define SYMHSS_ERR_TIMEOUT        -6  /* a bounded device wait expired */
#define SYMHSS_ERR_STATE          -7  /* calls out of order (e.g. factor before compress) */
#define SYMHSS_ERR_DEVICE         -8  /* a kernel detected an out-of-range index and skipped it */

/* ---- enums ---------------------------------------------------------------- */
#define SYMHSS_SYM     0   /* symmetric single-ID compression, row-scaled system (Eq. 15) */
#define SYMHSS_NONSYM  1   /* non-symmetric two-ID baseline, unscaled system (Sec. 6)    */

#define SYMHSS_FP64    0   /* every stage in FP64 */
#define SYMHSS_MIXED   1   /* FP64 compression; complex64 factorisation; FP64 refinement */

#define SYMHSS_MULLER  0   /* symmetric Muller-like system (Eq. 15): the method            */
#define SYMHSS_PMCHWT  1   /* symmetric PMCHWT comparator (Eq. symmetric_pmchwt): first order */
#define SYMHSS_BM      2   /* Burton-Miller comparator (Eq. bm): non-symmetric, first order;
                            * requires SYMHSS_NONSYM */

#define SYMHSS_HOST    0   /* pointer location flags */
#define SYMHSS_DEVICE  1

typedef struct symhss_s* symhss_t;  /* opaque handle */
typedef struct symhss_mlp_s* symhss_mlp_t;  /* opaque handle of a proposer network */

/* Sampled curve (Sec. 3.1): nodes gamma(theta_j) at theta_j = 2 pi j / n,
 * outward unit normals (pointing into the exterior Omega_0), trapezoidal
 * weights w_j = |gamma'(theta_j)| 2 pi / n and signed curvature kappa_j (positive
 * on a convex curve).  Equispaced parameters are required: the one-point
 * corrected diagonal relies on them.  Arrays have n doubles each and live in
 * host or device memory as `location` says; they are copied at create time. */
typedef struct {
  int n;
  const double *x, *y, *nx, *ny, *w, *kappa;
  int location;
} symhss_curve;

/* Solver parameters.  symhss_params_default fills the defaults shown. */
typedef struct {
  double k0, k1;          /* exterior / interior wavenumber (> 0)                   */
  double eps0, eps1;      /* material constants (> 0); eps_i = (k_i/omega)^2 (Sec. 2) */
  double tol;             /* relative ID tolerance |R_kk| <= tol |R_00|  (1e-10)      */
  int leaf;               /* leaf box size in nodes (128)                             */
  int nproxy;             /* minimum proxy points per ring (64)                       */
  double proxy_factor;    /* proxy ring radius / box radius (1.5)                     */
  int mode;               /* SYMHSS_SYM or SYMHSS_NONSYM                              */
  int precision;          /* SYMHSS_FP64, or SYMHSS_MIXED: the block LUs and the solves of the
                           * factorisation in complex64 (FP32: 60x the FP64 rate of the
                           * B300), the solution refined against the FP64 compressed operator
                           * (symhss_matvec): x <- x + B^{-1} (f - A x), 2 steps by default
                           * (symhss_set_refinement)                                        */
  int fixed_rank_kL;      /* > 0: fixed ranks k_l = ceil(a^(L-l) kL) (Sec. 4.3), 0: tol */
  double rank_scale_a;    /* a of Sec. 4.3 (1.15)                                     */
  int oversample;         /* sketch oversampling p (16): an ID is taken of Y = Omega M with
                           * s = rank estimate + p rows (+ 16 held-out rows) when that is
                           * under 0.8 m rows; an ID whose rank reaches s - p/2, or whose
                           * residual on the held-out rows exceeds tol, is redone on M;
                           * 0 disables the sketch */
  int formulation;        /* SYMHSS_MULLER (0) or the SYMHSS_PMCHWT comparator: row-scaled
                           * (SYMHSS_SYM) A = [-(e0 S0 + e1 S1), D0 + D1; D*0 + D*1,
                           * -(N0/e0 + N1/e1)], rhs [-W u_in; (1/e0) W du_in/dnu]; its
                           * hypersingular diagonal is one-point corrected (first order).
                           * SYMHSS_NONSYM gives the unscaled PMCHWT with two IDs.
                           * SYMHSS_BM (with SYMHSS_NONSYM only): rows [-e0 S0 - a e0 (D*0 + I/2),
                           * D0 - I/2 + a N0; -e1 S1, D1 + I/2], a = i/k0, rhs
                           * [-u_in - a du_in/dnu; 0], unscaled, two IDs.                 */
  uint64_t seed;          /* seed of the counter-based sketch generator               */
} symhss_params;

/* Per-handle statistics of the last compress / factor / solve. */
#define SYMHSS_MAX_LEVELS 32
/* kernel classes of the per-class device timing in symhss_stats_t */
#define SYMHSS_K_TILES  0   /* kernel-entry tile generator                       */
#define SYMHSS_K_ID     1   /* pivoted-QR column ID                              */
#define SYMHSS_K_GETRF  2   /* batched block LU                                  */
#define SYMHSS_K_GETRS  3   /* batched triangular solves (X = D^-1 L, Atilde, g)  */
#define SYMHSS_K_OTHER  4   /* bases, R X, small GEMMs, copies, gather / scatter  */
#define SYMHSS_K_SKETCH 5   /* tensor-core sketch Y = Omega M (slicing + tcgen05 GEMM) */
#define SYMHSS_K_CHECK  6   /* residual check of sketched IDs on held-out sketch rows  */
#define SYMHSS_K_MLP    7   /* proposer: box features + MLP forward                     */
#define SYMHSS_K_COUNT  8
/* In a batch: n and nboxes_leaf are totals, depth and root_size maxima, and the
 * level statistics cover level l of every problem that has it. */
typedef struct {
  int n;                          /* nodes                                    */
  int depth;                      /* L: leaves are at level L, root at 0       */
  int nboxes_leaf;
  int root_size;                  /* order of the root diagonal block          */
  int max_rank[2];                /* largest column-ID rank, flux / trace part */
  int level_max_rank[SYMHSS_MAX_LEVELS][2];
  double level_mean_rank[SYMHSS_MAX_LEVELS][2];
  int level_nproxy[SYMHSS_MAX_LEVELS];  /* proxy points per ring (max over boxes) */
  double ms_compress, ms_factor, ms_solve;  /* device time of the last call      */
  double ms_tiles, ms_id, ms_lu, ms_basis;  /* device time split of compress+factor */
  long long pairs_evaluated;      /* (point, point) kernel pairs of compress+factor */
  long long id_count;             /* interpolative decompositions performed     */
  double flops_lu;                /* real flops of block LU + solves in factor  */
  double flops_id;                /* real flops of the pivoted QRs              */
  long long device_bytes;         /* device memory held by the handle           */
  /* per kernel class, accumulated over the last compress + factor + solve: device
   * time from CUDA events recorded around each launch on the caller's stream,
   * number of launches, and algorithmic real flops (tiles: (point, point) pairs) */
  double kernel_ms[SYMHSS_K_COUNT];
  long long kernel_launches[SYMHSS_K_COUNT];
  double kernel_work[SYMHSS_K_COUNT];
  long long sketch_redo;          /* sketched IDs redone on the full matrix (rank near s
                                   * or residual check failed) */
  long long check_failed;         /* sketched IDs whose residual estimate exceeded tol  */
  double check_max_ratio;         /* largest accepted residual estimate ratio (<= tol)  */
  long long proposals;            /* ID ranks proposed by the attached network          */
  double proposal_rank_err;       /* mean |proposed - ID rank| / max(1, ID rank)        */
  long long proposal_under;       /* proposals below the ID rank                        */
  double ms_build;                /* device time of the last symhss_build                */
} symhss_stats_t;

/* ---- handle lifecycle ------------------------------------------------------ */

/* Fill `p` with the defaults above (k0 = k1 = 1, eps0 = eps1 = 1). */
int symhss_params_default(symhss_params* p);

/* Create a solver for `curve` with parameters `prm`.  Validates every input
 * (n >= 2, positive wavenumbers, material constants, weights; finite
 * coordinates; 1 <= leaf; nproxy >= 8; proxy_factor > 1; tol >= 0), copies the
 * curve, builds the box tree and proxy rings, and uploads them on `stream`.
 * On success *out owns all library allocations. */
int symhss_create(const symhss_curve* curve, const symhss_params* prm, void* stream, symhss_t* out);

/* Replace the node arrays by a new curve with the same n (same tree shape).
 * Invalidates any previous compression.  Single-problem handles only. */
int symhss_set_curve(symhss_t h, const symhss_curve* curve, void* stream);

/* A batch of `count` independent scatterers in one handle (many obstacles of
 * uneven size solved together; each is the problem of Sec. 2 on its own curve).
 * curves[c] and prms[c] describe problem c: wavenumbers and material constants
 * (k0, k1, eps0, eps1) may differ between problems; every other field of prms[c]
 * must equal that of prms[0] (else SYMHSS_ERR_INVALID).  Each problem gets its
 * own tree; compress / factor / solve then process the boxes of every problem at
 * the same tree height (counted from the leaves) together, one launch per kernel
 * and height, so the launch count follows the tallest tree, not the batch size.
 * Batch vectors (rhs, x of symhss_solve) stack the problems' [eq1; eq2] blocks in
 * problem order: problem c occupies rows [row0_c, row0_c + 2 n_c) with
 * row0_c = 2 (n_0 + ... + n_(c-1)), and a column has 2 (n_0 + ... + n_(count-1))
 * entries.  symhss_create is the count = 1 case.  The batch size is bounded by
 * device memory only (about the sum of the single-problem footprints). */
int symhss_create_batch(const symhss_curve* curves, const symhss_params* prms, int count, void* stream,
                        symhss_t* out);

/* Replace every problem's curve (same count and same n per problem). */
int symhss_set_curves(symhss_t h, const symhss_curve* curves, int count, void* stream);

/* Batch layout: *count problems (if count != NULL); n[c] nodes, depth[c] tree
 * depth and row0[c] first row of its block in batch vectors, for each array that
 * is not NULL (each with room for the problem count). */
int symhss_batch_info(symhss_t h, int* count, int* n, int* depth, long long* row0);

/* Proxy-method compression of every level (Sec. 4.1): kernel tiles M_R, one
 * column ID per box and component (two more row IDs of M_L per box with
 * SYMHSS_NONSYM).  Synchronises `stream` once per level to read ranks. */
int symhss_compress(symhss_t h, void* stream);

/* Multilevel factorisation (Sec. 4.2): block LU of every diagonal block,
 * X = D^{-1} L, Atilde = (R X)^{-1}, parent blocks, root LU.  Requires compress. */
int symhss_factor(symhss_t h, void* stream);

/* symhss_compress followed by symhss_factor, pipelined over tree heights: height t is
 * factorised on `stream` while height t + 1 is compressed on a high-priority stream the
 * handle owns (each height's factorisation needs only its own compression and the
 * factors one height down), so the latency-bound upper-level compression overlaps the
 * factorisation of the lower levels.  Same results as the two calls; stats().ms_build is
 * its device time (ms_compress and ms_factor are set to 0; per-kernel-class times are
 * summed over both streams).  Later work on `stream` is ordered after it. */
int symhss_build(symhss_t h, void* stream);

/* Right-hand side of the handle's system for the plane wave
 * u_in = exp(i k0 (x cos(angle) + y sin(angle))): [-eps0 W u_in ; W du_in/dnu]
 * (Eq. 15; PMCHWT: [-W u_in ; (1/eps0) W du_in/dnu]; Burton-Miller: [-u_in - (i/k0)
 * du_in/dnu ; 0]; the unscaled forms without W for SYMHSS_NONSYM).  rhs: device
 * complex128[2n] (a batch: every problem's block with its own k0 and eps0). */
int symhss_rhs_plane_wave(symhss_t h, double angle, void* rhs, void* stream);

/* Solve A x = rhs for `nrhs` right-hand sides (Sec. 4.2).  rhs, x: device
 * complex128[2n * nrhs], column j at offset 2n*j; rhs is not modified; rhs and x
 * may not overlap.  Requires factor. */
int symhss_solve(symhss_t h, const void* rhs, void* x, int nrhs, void* stream);

/* y = A_hss x: the handle's FP64 compressed operator (leaf diagonal blocks, sibling skeleton
 * blocks and the ID interpolation operators of every level, Sec. 4.1) applied to `nrhs`
 * vectors (device complex128[2n * nrhs], the layout of symhss_solve; x and y may not
 * overlap).  Requires factor (which keeps the operator's blocks).  Error to the exact
 * matrix: the compression's (about tol). */
int symhss_matvec(symhss_t h, const void* x, void* y, int nrhs, void* stream);

/* Refinement steps of SYMHSS_MIXED solves (0..4; 2 after create).  Each step applies
 * symhss_matvec and one more solve with the complex64 factors; each step gains a factor of
 * about kappa * 1e-7 (one step suffices at 2048 nodes, k 20/30; two at 65536 nodes, k 40/60). */
int symhss_set_refinement(symhss_t h, int steps);

/* As symhss_solve with host buffers: copies rhs in and x out inside the call. */
int symhss_solve_host(symhss_t h, const void* rhs_host, void* x_host, int nrhs, void* stream);

/* Statistics of the last phases (device-synchronising). */
int symhss_stats(symhss_t h, symhss_stats_t* out);

/* Column-ID ranks of level `level` (1..depth) of the first problem: out[2*b + h]
 * for box b and part h.  `out` is a host int array of 2 * 2^level entries. */
int symhss_level_ranks(symhss_t h, int level, int* out);

/* As symhss_level_ranks for problem `problem` of a batch (level 1..depth[problem]). */
int symhss_problem_ranks(symhss_t h, int problem, int level, int* out);

/* Largest ID rank the caller accepts (<= 0: no limit, the default).  A compression whose
 * column (or, with SYMHSS_NONSYM, row) ID of any box exceeds it stops with
 * SYMHSS_ERR_RANK_OVERFLOW and leaves the handle uncompressed; the handle stays usable (raise
 * the limit and compress again).  For callers that size later storage -- skeleton sets,
 * factors, transfers to other processes -- from a rank bound fixed in advance. */
int symhss_set_rank_limit(symhss_t h, int max_rank);

/* Device-memory budget, in bytes, for the buffers the handle allocates or grows in its later
 * calls (<= 0: none, the default).  An allocation that would take the handle's total beyond
 * it fails before cudaMalloc is called, and the call returns SYMHSS_ERR_NOMEM as on a full
 * device; the handle stays usable and a later call succeeds once the budget allows.  For
 * callers that share one GPU between several solvers under a fixed memory plan.  Buffers
 * allocated by symhss_create are not counted. */
int symhss_set_memory_limit(symhss_t h, long long bytes);

/* Release everything the handle owns.  NULL is accepted. */
int symhss_destroy(symhss_t h);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles and entry points; for launch accounting in benchmarks). */
long long symhss_launch_count(void);

/* Static message for a status code. */
const char* symhss_strerror(int status);

/* ---- launch tuning and the autotuner -------------------------------------------------
 * Launch-shape choices that do not change any result bit (tile_loop_chunk and id_cluster_max
 * change nothing either: the same arithmetic runs in other blocks), and lu_tc, which selects
 * the factorisation's arithmetic path. */
typedef struct {
  int lu_lookahead;       /* 1: next LU panel on a high-priority stream during the trailing update */
  int lu_panel_threads;   /* 256, 512 or 1024: largest thread block of the LU panel kernel      */
  int tile_loop_chunk;    /* 0: adaptive (8..32 by launch size); else 8, 16 or 32 loop points per block */
  int id_cluster_max;     /* 1, 2, 4, 8 or 16: largest thread-block cluster of one column ID      */
  int lu_panel_cluster;   /* 1, 2, 4, 8 or 16 (default 16): largest thread-block cluster factoring
                           * one LU panel, used while blocks x cluster <= the SM count and every
                           * member keeps >= 32 panel rows (the top tree levels); 1: one block */
  int lu_tc;              /* 1 (default): FP64 block LUs blocked by lu_outer columns and multi-RHS
                           * solves blocked by 64 rows, their updates on the tensor cores
                           * (symhss_zgemm); 0: 16-column LU and unblocked solves on the FP64
                           * pipe; 2: the first for launches of at least 32 blocks (the lower tree
                           * levels; solves also when blocks x right-hand sides >= 512), the second
                           * above.  All give the factorisation to FP64 rounding, not the same bits. */
  int lu_outer;           /* column block of the LU's tensor-core updates: 16 (default), 32 or 64
                           * (0 = 64); 16: a rank-16 update on the tensor cores after every
                           * 16-column panel, no FP64 updates inside a block.  The blocked
                           * solves keep 64-row blocks (measured faster than 16 or 32). */
  int reserved[1];
} symhss_tuning;

int symhss_get_tuning(symhss_t h, symhss_tuning* out);
/* Set the handle's launch tuning (values outside the lists above: SYMHSS_ERR_INVALID). */
int symhss_set_tuning(symhss_t h, const symhss_tuning* t);
/* Autotuner: time the handle's own compress / factor with each value of each tunable
 * (coordinate search: tile_loop_chunk and id_cluster_max on compress, then lu_tc x lu_outer
 * (block LU + solve time), lu_panel_threads x lu_lookahead, then lu_panel_cluster x
 * lu_lookahead on factor), `reps` runs
 * per value, the minimum device time of the affected kernel classes deciding; leaves the best
 * tuning set (and in *out, if not NULL) and the handle compressed and factorised.
 * Synchronises `stream`. */
int symhss_autotune(symhss_t h, int reps, symhss_tuning* out, void* stream);

/* ---- learned rank / skeleton proposer (an addition to the paper's method) --------------
 * A 3-layer MLP (128 inputs, two hidden layers of 128 with ReLU, 128 outputs of which
 * 66 are used), FP16 weights with FP32 accumulation; FP32 master weights and Adam state
 * for training.  Parameters are packed float[SYMHSS_MLP_PARAMS]:
 * [W1 (128 x 128 row-major, out x in), b1, W2, b2, W3, b3].  Inputs are the 128 box
 * features of symhss_training_data; output 0 / 1 is log2(1 + rank) / 8 of the box's
 * flux / trace column ID, outputs 2..33 / 34..65 skeleton logits at 32 positions along
 * the box.  Training loss over B boxes: (1/B) sum (o_h - y_h)^2
 * + (0.1 / 64B) sum mask * BCE(sigmoid(o), t). */
#define SYMHSS_MLP_PARAMS 49536
#define SYMHSS_MLP_WIDTH  128

/* Create a network holding `params` (host float[SYMHSS_MLP_PARAMS]; NULL = zeros) with
 * scratch for batches of up to max_batch samples (device-synchronising). */
int symhss_mlp_create(const float* params, int max_batch, symhss_mlp_t* out);
/* Replace the master weights (host array; NaN/Inf refused) and reset the Adam state. */
int symhss_mlp_set_params(symhss_mlp_t net, const float* params);
/* Copy the FP32 master weights (params) and/or their FP16 copy (fp16_params, 2-byte
 * IEEE halves) to host arrays; either may be NULL. */
int symhss_mlp_get_params(symhss_mlp_t net, float* params, void* fp16_params);
/* out[b, :] = network(x[b, :]) for `batch` samples (device float arrays, row-major
 * batch x 128; any batch size). */
int symhss_mlp_forward(symhss_mlp_t net, const float* x, int batch, float* out, void* stream);
/* Loss and its gradient with respect to the FP16 weights for one batch (<= max_batch):
 * x batch x 128, y_rank batch x 2, y_skel and mask batch x 64 (device float arrays);
 * loss (host double) and grad (host float[SYMHSS_MLP_PARAMS]) may be NULL. */
int symhss_mlp_loss_grad(symhss_mlp_t net, const float* x, const float* y_rank, const float* y_skel,
                         const float* mask, int batch, double* loss, float* grad, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on one batch; the FP16
 * copy is refreshed from the master weights.  loss (host) may be NULL (no sync). */
int symhss_mlp_train_step(symhss_mlp_t net, const float* x, const float* y_rank, const float* y_skel,
                          const float* mask, int batch, float lr, double* loss, void* stream);
int symhss_mlp_destroy(symhss_mlp_t net);

/* Attach a trained network to a solver handle (NULL detaches; the network must outlive
 * its use).  During symhss_compress the network proposes each box's two ID ranks r~ and
 * the randomized sketch of that ID gets s = 16 ceil((ceil(margin r~) + 2 + oversample) / 16)
 * rows for the ID (at least 32) instead of the default estimate.  While a network is
 * attached, every sketched ID is accepted only if its interpolation residual on the proxy
 * matrix itself, max_c ||m_c - M_J t_c||, is at most tol times the largest column norm of M
 * (the bound the plain ID meets by construction); an ID that fails continues its pivoted QR
 * on the sketch at tol / 16 and is checked again, and is otherwise redone as a plain ID of
 * the proxy matrix.  (Without a network the check uses 16 held-out sketch rows, an
 * a-posteriori estimate of that residual.)  margin >= 1.  Has no effect with oversample = 0
 * or fixed ranks. */
int symhss_set_proposer(symhss_t h, symhss_mlp_t net, double margin);

/* Training data of the last compression: one sample per compressed (non-root) box of
 * every problem, ordered by tree height, problem, box.  *count: in = capacity of the
 * arrays (ignored when x is NULL), out = number of boxes (all arrays may be NULL to query
 * the count).  x: count x 128 features; y_rank: count x 2 (log2(1 + rank) / 8); y_skel,
 * mask: count x 64 skeleton fractions and position masks; meta: count x 10 ints
 * (problem, level, height, first node within the problem, node count, active flux and
 * trace counts, near rows, proxy points, 0); geo: count x 3 (box centre x, y, radius).
 * Host arrays; requires compress. */
int symhss_training_data(symhss_t h, int* count, float* x, float* y_rank, float* y_skel, float* mask, int* meta,
                         double* geo, void* stream);

/* ---- building blocks (device pointers; used by the solver, exposed for tests) ---- */

/* H_0^(1)(x_i) and H_1^(1)(x_i) (Sec. 3.1: G_k = (i/4) H_0(k r)) for n device doubles
 * x_i > 0, written to out (device complex128[2n]): H_0 values, then H_1 values.
 * The evaluator the tile generator uses (power series, Miller's recurrence,
 * Hankel's expansion; about 1e-15 relative accuracy). */
int symhss_hankel01(const double* x, int n, void* out, void* stream);

/* The reciprocal the LU panels (Sec. 4.2 factorisation) take of each pivot: out_i ~ 1 / a_i
 * for n device complex128 values a (out: device complex128[n]), as conj(a) / |a|^2 with
 * 1 / |a|^2 from Newton's iteration for the reciprocal (two steps from the hardware's
 * approximation), or by Smith's scaled division when |a|^2 is outside [2^-996, 2^997).
 * Within a few units in the last place of 1 / a; zero gives non-finite values. */
int symhss_pivot_reciprocal(const void* a, int n, void* out, void* stream);

/* A set of points for symhss_kernel_block: coordinates, unit normals, weights,
 * curvature and an id; two points with the same id >= 0 are the same curve
 * node and receive the corrected diagonal (Sec. 3.1) and the free terms (Eq. 15).
 * hs: each node's speed term of the hypersingular diagonal (symhss_speed_terms of
 * its curve's weights), used only by the PMCHWT and Burton-Miller diagonals; NULL
 * reads as zero (a circle).  All arrays are device arrays of n entries. */
typedef struct {
  int n;
  const double *x, *y, *nx, *ny, *w, *kappa;
  const int* id;
  const double* hs;
} symhss_points;

/* Speed term of the one-point corrected hypersingular diagonal (Sec. 3.1, used by the
 * PMCHWT and Burton-Miller comparators) for one closed curve given by its n trapezoidal
 * weights w_j = |gamma'(theta_j)| 2 pi / n (host arrays; w > 0 and finite, else
 * SYMHSS_ERR_INVALID).  The hypersingular kernel times the source's speed v = |gamma'| has
 * the constant term v [kappa^2 / (24 pi) + (v''/6 - v'^2/(4 v)) / (2 pi v^3)] about a node;
 * the second part equals s_j / w_j^2 with
 *   s_j = ((d2w_j / w_j) / 6 - (d1w_j / w_j)^2 / 4) / (2 pi),
 * d1w, d2w the first and second derivatives of the periodic sequence w with respect to the
 * index j, taken by central differences of order 16 (fewer points for n < 17).  Writes s
 * (host double[n]; zero on a circle).  Handles compute it from their curves at create. */
int symhss_speed_terms(const double* w, int n, double* s);

/* Tile generator: out[i + j*ld] = A[(obs_i, obs_eq[i]), (src_j, src_comp[j])]
 * with eq/comp in {0, 1} (0: first equation / flux unknown q, 1: second
 * equation / trace unknown u).  `scaled` = 1 gives the row-scaled symmetric
 * matrix (Eq. 15), 0 the unscaled baseline (Sec. 6).  out: device complex128,
 * column-major, ld >= obs->n. */
int symhss_kernel_block(const symhss_params* prm, const symhss_points* obs, const int* obs_eq,
                        const symhss_points* src, const int* src_comp, int scaled,
                        void* out, int ld, void* stream);

/* Batched column interpolative decomposition (Sec. 4.1) by Householder QR with
 * column pivoting: for each of `batch` matrices M_b = A + b*strideA (m x n,
 * column-major, leading dimension lda, complex128, OVERWRITTEN), find rank r_b,
 * a permutation perm_b (n ints at perm + b*n) and T_b = R11^{-1} R12 (r_b x (n-r_b),
 * column-major with leading dimension r_b, at T + b*strideT complex128 entries;
 * strideT >= floor(n/2)*ceil(n/2) always suffices) with
 * M_b[:, perm_b] ~= M_b[:, perm_b[:r_b]] [I T_b].
 * fixed_rank < 0: stop at the first |R_kk| <= tol |R_00|; else exactly
 * min(fixed_rank, m, n) steps.  rank: device int[batch]. */
int symhss_column_id(void* A, int m, int n, int lda, long long strideA, int batch, double tol,
                     int fixed_rank, int* rank, int* perm, void* T, long long strideT, void* stream);

/* symhss_column_id for callers that cannot allocate device memory: same
 * arguments, results and errors, but no cudaMalloc / cudaFree (or any other
 * allocating call) is made.  Such callers are, e.g., code running under a fixed
 * device-memory budget or inside an allocator it does not own, and latency-
 * critical loops that cannot afford the implicit device-wide synchronisation of
 * cudaMalloc / cudaFree.  The scratch it needs (job descriptors, reference norms,
 * a status word) lives in one library-owned __device__ array sized for at most
 * 4096 matrices per call, which every GPU that loads the library keeps until the
 * process exits; batch > 4096 returns SYMHSS_ERR_INVALID.  The first call on a
 * device looks up that array's device address with the device current; the
 * address is kept for the process, so the device must not be reset
 * (cudaDeviceReset) while the library is in use.  Every call synchronises
 * `stream` to read its status word back, so no call can be made while the stream
 * is being captured into a graph.  Every call reuses the same array: calls
 * whose GPU work overlaps (unordered streams or host threads) race and must not
 * be issued.  This entry point is an engineering addition with no counterpart in
 * the paper. */
int symhss_column_id_noalloc(void* A, int m, int n, int lda, long long strideA, int batch, double tol,
                             int fixed_rank, int* rank, int* perm, void* T, long long strideT, void* stream);

/* Randomized row sketch Y_b = Omega_b M_b on the tensor cores, to FP64 accuracy
 * (the sketch of the randomized ID; the ID of Y_b selects the columns of M_b).
 * M_b = A + b*strideA: m x n complex128, column-major, leading dimension lda (read
 * only).  Omega_b is the s x m matrix with entries -1 where the top bit of
 * splitmix64(seed ^ b*0xD1B54A32D192ED03 ^ i*0x8CB92BA72F3D8DD7 ^ k) is set and +1
 * otherwise (i: row of Y, k: row of M; 64-bit wrapping arithmetic).  Y_b = Y +
 * b*strideY: s x n complex128, leading dimension ldy.  m <= 65536, s <= 1024.
 * Returns SYMHSS_ERR_TIMEOUT if a bounded device wait expired (see
 * symhss_set_wait_limit_ns); Y is then undefined but the device stays usable. */
int symhss_sketch(const void* A, int m, int n, int lda, long long strideA, int batch, int s,
                  unsigned long long seed, void* Y, int ldy, long long strideY, void* stream);

/* Time limit, in nanoseconds, of each bounded wait inside the tensor-core kernels (the
 * sketch's waits for its bulk copies and MMAs, the matrix product's waits for its MMAs) for
 * launches made after this call, process-wide; ns <= 0 restores the default of 200 ms.  When
 * a wait expires the kernel records the timeout, waits once more (bounded by the default)
 * for the copies or MMAs it may still have in flight, frees its tensor memory and exits; the
 * call (symhss_sketch, symhss_zgemm, or a solver call that runs them) returns
 * SYMHSS_ERR_TIMEOUT and the CUDA context stays usable.  Intended for exercising that path
 * in tests; a very short limit makes every such kernel time out. */
int symhss_set_wait_limit_ns(long long ns);

/* Test hook for the timeout path of the tensor-core matrix product (symhss_zgemm and the
 * factorisation's blocked LU and solves, which use it): while on (on != 0), the last wait
 * of every product launch waits for an mbarrier phase that no commit completes, so it
 * expires after the wait limit (symhss_set_wait_limit_ns); the kernel then waits for its
 * MMAs in flight, frees its tensor memory and the call returns SYMHSS_ERR_TIMEOUT with the
 * CUDA context usable.  Off after load; process-wide. */
int symhss_set_timeout_probe(int on);

/* Batched complex FP64 matrix product on the tensor cores: for b < batch,
 *   mode 0: C_b = A_b B_b,   mode 1: C_b -= A_b B_b,   mode 2: C_b += A_b B_b,
 * A_b = A + b*strideA (m x k, leading dimension lda), B_b = B + b*strideB (k x n, ldb),
 * C_b = C + b*strideC (m x n, ldc); complex128, column-major, device pointers; C must not
 * overlap A or B.  This is the product the factorisation (Sec. 4.2) applies to its
 * diagonal blocks: each row of A and each column of B is scaled by its largest power of two
 * and cut into eight 7-bit slices that are exact in bf16; the 36 slice products of weight
 * at least 2^-49 are summed exactly in FP32 on the tcgen05 tensor cores and recombined in
 * integers, so every entry is within about 2^-52 k max_l |A(i,l)| max_l |B(l,j)| of the
 * exact product (the usual FP64 bound with row and column maxima).  k > 64 is split into
 * chunks of 64 accumulated in FP64.  Returns SYMHSS_ERR_TIMEOUT if a bounded device wait
 * expired (symhss_set_wait_limit_ns). */
int symhss_zgemm(const void* A, int lda, long long strideA, const void* B, int ldb, long long strideB, void* C,
                 int ldc, long long strideC, int m, int n, int k, int batch, int mode, void* stream);

/* Batched LU with partial pivoting of n x n complex128 matrices A + b*strideA
 * (leading dimension lda; overwritten by L\U), pivots ipiv + b*n (0-based row
 * swapped with row k at step k), info[b] = 0 or k+1 for the first zero pivot. */
int symhss_lu_batched(void* A, int n, int lda, long long strideA, int batch, int* ipiv,
                      int* info, void* stream);

/* Solve with the factors of symhss_lu_batched: B_b <- A_b^{-1} B_b for nrhs
 * columns (leading dimension ldb, stride strideB). */
int symhss_lu_solve_batched(const void* LU, int n, int lda, long long strideA, const int* ipiv,
                            void* B, int nrhs, int ldb, long long strideB, int batch, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SYMHSS_H */
