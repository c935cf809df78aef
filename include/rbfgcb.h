/*
 * rbfgcb.h -- C ABI of librbfgcb.so: GB300 (sm_103a) kernels for RBF mesh
 * deformation with the grouping-circular-based (GCB) greedy selection of
 * support nodes (arXiv:2004.04817).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Point and displacement arrays are row-major n x 3 (x, y, z per row),
 *    unless a signature says otherwise.
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; the
 *    caller owns them (allocates, frees, keeps them alive until the stream
 *    work completes).  Pointers named h_* are HOST pointers.  The library never
 *    frees caller memory.
 *  - Scratch comes from the caller-supplied device workspace `d_ws` of
 *    `ws_bytes` bytes, sized with the matching *_workspace_bytes query; the
 *    workspace must be 256-byte aligned.  Entry points allocate no device
 *    memory of their own.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every call returns an rbf_status; argument errors are reported before any
 *    work is enqueued.  Calls marked SYNCHRONOUS block until their stream work
 *    is done (their outputs include host scalars).  Calls marked ASYNC only
 *    enqueue; device-side failures of an ASYNC call are reported by the next
 *    SYNCHRONOUS call or by rbf_last_device_status().
 *  - No call falls back to the CPU.  Without a usable CUDA device every call
 *    returns RBF_E_CUDA.
 *
 * Notation (paper): boundary nodes r_j with prescribed displacements dr_j
 * (N_b of them), support set S (N_c nodes), support radius R, Wendland C2
 * basis phi(eta) = (1 - eta)^4 (4 eta + 1) for eta = |r - r_j| / R < 1 and 0
 * otherwise (Eq. 2), interpolant F(r) = sum_{j in S} w_j phi(|r - r_j| / R)
 * (Eq. 1), weights from Phi_SS W = dX_S (Eqs. 3-5), interpolation error of a
 * boundary node E_q = |dr_q - F(r_q)|_2.
 */
#ifndef RBFGCB_H
#define RBFGCB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RBF_OK = 0,
    RBF_E_ARG = 1,        /* invalid argument (sizes, radius, m, alignment, NULL) */
    RBF_E_NOT_SPD = 2,    /* a Cholesky pivot d^2 <= 1e-13: coincident or nearly
                             coincident support nodes (Phi is SPD only for
                             distinct nodes, Sec. 2) */
    RBF_E_NC_MAX = 3,     /* the greedy wanted more than nc_max support nodes;
                             the partial selection is returned */
    RBF_E_NONFINITE = 4,  /* NaN or Inf in an input */
    RBF_E_WORKSPACE = 5,  /* workspace missing, too small or misaligned */
    RBF_E_TIMEOUT = 6,    /* a bounded device-side wait (grid barrier) ran out;
                             the kernel returned without finishing */
    RBF_E_CUDA = 7        /* a CUDA runtime call failed (no device, launch error) */
} rbf_status;

/* Precision of the pair evaluations (Eq. 1 sums). */
enum {
    RBF_PREC_F64 = 64,    /* every pair in FP64 */
    RBF_PREC_F32 = 32,    /* FP32 pairs; the greedy certifies its argmax and its
                             stopping test by re-scoring near-maximal nodes in
                             FP64 (FP32 values carry an error bound) */
    RBF_PREC_F32X2 = 48   /* double-float pairs on the FP32 pipe (about 44
                             correct bits); the greedy re-scores only nodes
                             within the double-float bound of the maximum in
                             FP64 */
};

typedef struct {
    double radius;        /* support radius R > 0 (eta = distance / R) */
    double tol;           /* E*; absolute, or relative (tol_mode = 1) */
    int32_t tol_mode;     /* 0: E* = tol; 1: E* = tol * max_j |dr_j|_2 */
    int32_t eval_prec;    /* RBF_PREC_F64, RBF_PREC_F32 or RBF_PREC_F32X2 */
    int64_t m;            /* number of groups, 1 <= m <= N_b (1 = plain greedy) */
    uint64_t seed;        /* seed of the random partition into groups */
    int64_t nc_max;       /* capacity of the support set, 3 <= nc_max <= N_b */
    int32_t refine_steps; /* FP64 iterative-refinement steps in rbf_solve_weights */
    int32_t flags;        /* 0, or RBF_FLAG_HISTORY_FULL */
    int32_t ctas;         /* rbf_greedy_select: CTAs of the persistent launch
                             (0 = chosen from the group size); tuning only */
    int32_t reserved;     /* must be 0 */
} rbf_params;

/* rbf_params.flags: with a history buffer, also evaluate all N_b errors in
 * FP64 after every m-th iteration to fill its global max / RMS columns
 * (diagnostic; the selection does not depend on it). */
#define RBF_FLAG_HISTORY_FULL 1
/* rbf_params.flags, tests of the failure path only: one CTA of the
 * persistent greedy kernel leaves before its first grid barrier and every
 * barrier wait is bounded by 50 ms, so rbf_greedy_select returns
 * RBF_E_TIMEOUT (and the CUDA context stays usable). */
#define RBF_FLAG_TEST_BARRIER_TIMEOUT (1 << 30)

/* Per-run statistics of rbf_greedy_select (host struct). */
typedef struct {
    int64_t iterations;      /* greedy iterations run (k - 3 + 1 at exit)      */
    int64_t nc;              /* |S| at exit                                     */
    int64_t full_checks;     /* all-node evaluations: history checks and the
                                look-aheads over idle runs                     */
    int64_t pairs_f32;       /* (node, centre) pairs evaluated in FP32          */
    int64_t pairs_f64;       /* (node, centre) pairs evaluated in FP64          */
    int64_t pairs_ff;        /* (node, centre) pairs evaluated in double-float  */
    int64_t rescored;        /* nodes re-scored in FP64 after an FP32 screen    */
    double estar;            /* the absolute tolerance E* used                  */
    double final_max;        /* certified global max error at exit: the FP64
                                maximum (FP64 mode, or where the last check
                                re-scored in FP64), else the largest certified
                                upper bound E~ + beta of the screened errors
                                (>= the maximum, <= E* at a normal exit);
                                -1 if the run ended on an error status        */
    double final_rms;        /* RMS error over the nodes outside S at exit, a
                                diagnostic summed in FP32 (about 1e-6
                                relative); in the screened modes nodes not
                                re-scored enter with their screened value (-1
                                on an error status)                            */
    double min_pivot;        /* smallest squared Cholesky pivot d^2 seen        */
    double max_resid;        /* with d_w: max_j |F(r_j) - dr_j|_inf over S after
                                refinement (FP64); -1 without d_w             */
    int64_t phase_ns[12];    /* device time of the persistent kernel's first CTA
                                by phase: [0] prologue (packing, seeds),
                                [1] evaluation bookkeeping, [2] FP64
                                re-scores, [3] appends, [4] final refinement,
                                [5] other, [6] of all that, time spent waiting
                                in grid barriers, [7] centre staging, [8] error
                                pass, [9] block reductions, [10] evaluation
                                barrier + grid reduction, [11] error pass of
                                the look-aheads over all nodes                */
    int64_t barriers;        /* grid barriers the persistent kernel passed      */
    int64_t ctas;            /* CTAs that ran this problem                      */
} rbf_greedy_stats;

/* Columns of one row of the optional iteration history (device doubles):
 * [k, |S| before the step, local max E in G_(k mod m), global max E (or -1 if
 *  no full check ran), global RMS E (or -1), node added (or -1)]. */
#define RBF_HIST_COLS 6

/* --------------------------------------------------------------------------
 * Greedy / GCB support-node selection (Sec. 3, Algorithm 1; m = 1 is the
 * plain Rendall-Allen greedy of Sec. 1).
 *
 * Partition: node perm[p] of a SplitMix64-driven Fisher-Yates permutation
 * belongs to group p mod m (groups disjoint, covering, sizes within one,
 * Sec. 3).  Seed nodes: n0 = argmax |dr_j|, n1 = the node farthest from n0,
 * n2 = the node farthest from {n0, n1} (lowest index on ties).  Iteration k
 * (from 3) evaluates E_q for q in G_(k mod m) minus S with the current
 * weights, takes the largest FP64 E_q (the lowest index only among exactly
 * equal values) and appends it to S when E > E* (strict).  The Cholesky factor of Phi_SS grows by one row per
 * appended node (recurrence Cholesky, Sec. 1), in FP64.  The run stops after
 * m consecutive iterations without an append: those m groups cover every
 * node (Sec. 3) and share one set of weights, so max_q E_q <= E* is then
 * certified (in FP32 mode every decision uses FP64 values: the FP32 errors
 * carry a bound, and each node whose bound reaches the group maximum is
 * re-scored in FP64).
 *
 * d_xb, d_db : device FP64, nb x 3 (boundary coordinates, displacements).
 * d_sel_idx  : device int32[nc_max]: selected node indices in selection order
 *              (the three seed nodes first).
 * d_sel_iter : device int64[nc_max] or NULL: iteration k at which each node
 *              was added (-1 for seeds).
 * d_w        : device FP64 nc_max x 3 or NULL: the weights of the selected
 *              set (support order), from the greedy's own factor refined by
 *              p->refine_steps FP64 steps W += Phi_SS^-1 (dX_S - Phi_SS W) --
 *              the same result rbf_solve_weights gives, without refactoring.
 * d_hist     : device double[hist_cap * RBF_HIST_COLS] or NULL.
 * h_nc       : host; number of selected nodes.
 * h_n_hist   : host or NULL; number of iterations (history rows wanted).
 * h_stats    : host or NULL.
 * SYNCHRONOUS.  Returns RBF_E_NC_MAX with a valid partial selection when the
 * cap is reached, RBF_E_NOT_SPD when an append meets a non-positive pivot.
 * ------------------------------------------------------------------------ */
size_t rbf_greedy_workspace_bytes(int64_t nb, const rbf_params *p);

rbf_status rbf_greedy_select(const double *d_xb, const double *d_db, int64_t nb,
                             const rbf_params *p,
                             int32_t *d_sel_idx, int64_t *d_sel_iter, double *d_w,
                             double *d_hist, int64_t hist_cap,
                             int64_t *h_nc, int64_t *h_n_hist,
                             rbf_greedy_stats *h_stats,
                             void *d_ws, size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * Certified screening record of a finished greedy run (FP32 and double-float
 * modes; Alg. 1's argmax and E > E* test decide on these values).  After
 * rbf_greedy_select returned RBF_OK on workspace d_ws (same nb and p), every
 * boundary node outside S was last evaluated with the final weights of the
 * evaluation table; for each node n this gives that screened error E~_n
 * (d_err[n], FP64) and its bound beta_n (d_bound[n], FP32) with
 * |E~_n - E_n| <= beta_n, E_n the exact error with those weights (beta_n = 0
 * where an FP64 re-score replaced the screened value).  d_w_eval (nc x 3
 * FP64, nc = the run's N_c) receives the table's weights: the FP32 values
 * (FP32 mode) or the double-float sums h + l (double-float mode).  Entries
 * of nodes in S are stale.  The bounds are derived in the library's sources
 * (constants at the screened evaluation).  ASYNC.
 * ------------------------------------------------------------------------ */
rbf_status rbf_greedy_screen_errors(const void *d_ws, size_t ws_bytes, int64_t nb,
                                    const rbf_params *p, int64_t nc, double *d_err,
                                    float *d_bound, double *d_w_eval, void *stream);

/* --------------------------------------------------------------------------
 * Peak-selection variant of the greedy (the prior art the paper cites in
 * Sec. 1: several error-peak nodes added at a time).  In each iteration the
 * nodes of the active group outside S with E > E* are taken in decreasing E
 * (lowest node index on ties), each only if it lies at least `separation`
 * (absolute, the units of d_xb) from every node taken before it in the same
 * iteration, up to `peaks` nodes (1..16); they are appended in that order.
 * peaks = 1 is rbf_greedy_select.  The selection is exact: in the screened
 * precisions it is certified from the error bounds, or every candidate of
 * the group is re-scored in FP64 first.  Termination, partition, seeds and
 * outputs as rbf_greedy_select (no iteration history); several nodes share
 * an iteration number in d_sel_iter.  SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
rbf_status rbf_greedy_select_peaks(const double *d_xb, const double *d_db, int64_t nb,
                                   const rbf_params *p, int peaks, double separation,
                                   int32_t *d_sel_idx, int64_t *d_sel_iter, double *d_w,
                                   int64_t *h_nc, rbf_greedy_stats *h_stats, void *d_ws,
                                   size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * Batched greedy: many independent problems (for instance one wing per load
 * case or per design) in ONE cooperative launch.  Problem i runs Algorithm 1
 * as rbf_greedy_select would, on its own contiguous range of CTAs (at least
 * one; more for larger groups), with its own workspace segment, barrier and
 * control block, so problems of very different sizes proceed independently.
 *
 *   create  (SYNCHRONOUS, host work): validates, computes each problem's
 *           partition, assigns CTAs, writes per-problem arguments into d_ws;
 *           returns an opaque host handle (freed by destroy).
 *   run     (ASYNC, no host synchronisation or host-memory access, so it can
 *           be captured in a CUDA graph and replayed): resets the control
 *           blocks and launches the kernel.
 *   results (SYNCHRONOUS): status and statistics of every problem.
 *
 * All problems must share params.eval_prec; B <= number of co-resident CTAs.
 * d_sel_idx (int32[nc_max]) and d_w (FP64 nc_max x 3 or NULL) receive each
 * problem's selection and refined weights; rbf_greedy_batch_nc_device gives
 * the device array of |S| per problem (int64[B]) for rbf_volume_batch.
 * ------------------------------------------------------------------------ */
typedef struct {
    const double *d_xb;   /* device FP64 nb x 3 */
    const double *d_db;   /* device FP64 nb x 3 */
    int64_t nb;
    rbf_params params;
    int32_t *d_sel_idx;   /* device int32[params.nc_max] (output) */
    double *d_w;          /* device FP64 params.nc_max x 3 or NULL (output) */
    int64_t *d_sel_iter;  /* device int64[params.nc_max] or NULL (output): the
                             iteration k of Alg. 1 that appended each node
                             (-1 for the seed nodes), as rbf_greedy_select */
} rbf_greedy_problem;

typedef struct rbf_greedy_batch rbf_greedy_batch;

size_t rbf_greedy_batch_workspace_bytes(const rbf_greedy_problem *h_probs, int B);
rbf_status rbf_greedy_batch_create(const rbf_greedy_problem *h_probs, int B,
                                   void *d_ws, size_t ws_bytes, void *stream,
                                   rbf_greedy_batch **out);
rbf_status rbf_greedy_batch_run(rbf_greedy_batch *b, void *stream);
const int64_t *rbf_greedy_batch_nc_device(const rbf_greedy_batch *b);
rbf_status rbf_greedy_batch_results(rbf_greedy_batch *b, int32_t *h_status,
                                    rbf_greedy_stats *h_stats, void *stream);
void rbf_greedy_batch_destroy(rbf_greedy_batch *b);

/* --------------------------------------------------------------------------
 * Support weights: solve Phi_SS W = dX_S (Eqs. 4-5 restricted to S, SPD by
 * Sec. 2) in FP64 by a recurrence Cholesky, then p->refine_steps steps of
 * iterative refinement W += Phi_SS^-1 (dX_S - Phi_SS W) with the residual
 * recomputed from coordinates.
 *
 * d_sel_idx : device int32[nc], distinct indices into the nb boundary nodes.
 * d_w       : device FP64 nc x 3 (output weights, support order).
 * h_max_resid : host or NULL; max_j |F(r_j) - dr_j|_inf over j in S after
 *               refinement (FP64).
 * SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
size_t rbf_solve_workspace_bytes(int64_t nc);

rbf_status rbf_solve_weights(const double *d_xb, const double *d_db, int64_t nb,
                             const int32_t *d_sel_idx, int64_t nc,
                             const rbf_params *p, double *d_w,
                             double *h_max_resid,
                             void *d_ws, size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * General support system: solve Phi_SS X = B for a caller's right-hand side
 * (Eqs. 4-5 with B in place of dX_S), with the same FP64 factorisation and
 * refinement as rbf_solve_weights.  Used by the adjoint (Phi_SS is
 * symmetric, so Phi_SS^-T = Phi_SS^-1) and by the differentiable forward map.
 *
 * d_rhs : device FP64 nc x 3 (support order).   d_x : device FP64 nc x 3.
 * h_max_resid : host or NULL; max_j |(Phi_SS X - B)_j|_inf.
 * Workspace: rbf_solve_workspace_bytes(nc).  SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
rbf_status rbf_solve_system(const double *d_xb, int64_t nb, const int32_t *d_sel_idx,
                            int64_t nc, const double *d_rhs, const rbf_params *p,
                            double *d_x, double *h_max_resid,
                            void *d_ws, size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * Volume displacements, Eq. 6: dv_v = sum_{j in S} w_j phi(|x_v - r_j| / R)
 * for the nv volume points.
 *
 * d_xv : FP64 nv x 3.   d_dv : FP64 nv x 3 (output).  Both may be device
 *        memory or pinned host memory that the device reaches at the same
 *        address (on a GB300 the kernels then read the points and write the
 *        displacements over NVLink-C2C, each once, with no separate copy);
 *        any other pointer gives RBF_E_ARG before device work.
 * d_xb, d_sel_idx, nc, d_w : centres r_j = xb[sel_idx[j]] and weights w_j
 *                            (device FP64 nc x 3), as from rbf_solve_weights.
 * p->eval_prec selects the pair arithmetic (FP32, double-float or FP64); only
 * radius and eval_prec are read from p.
 * ASYNC.
 * ------------------------------------------------------------------------ */
size_t rbf_volume_workspace_bytes(int64_t nv, int64_t nc, const rbf_params *p);

rbf_status rbf_deform_volume(const double *d_xv, int64_t nv,
                             const double *d_xb, const int32_t *d_sel_idx,
                             int64_t nc, const double *d_w,
                             const rbf_params *p, double *d_dv,
                             void *d_ws, size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * Many displacement fields on one support set in double-float (Eq. 6 for
 * every column of W): D = Phi_vc W, W nc x n_out FP64 (row-major, support
 * order), e.g. n_out = 96 for 32 modes of 3 components.  phi is computed once
 * per (point, centre) pair in double-float and shared by all columns; the
 * products and sums are double-float on the FP32 pipe, so the result carries
 * FP64-level accuracy (about 2^-44 sum_j |w_j phi_vj| per column), unlike the
 * tensor-core path, whose FP32 accumulation limits it to about 2^-24 sum_j
 * |w_j phi_vj| -- too coarse when the weights of a support set cancel
 * heavily (large radius, high modes).
 * p: radius; eval_prec must be RBF_PREC_F32X2.  1 <= n_out <= 192.
 * d_out : device FP64 nv x n_out (row-major).  ASYNC.
 * ------------------------------------------------------------------------ */
size_t rbf_volume_fields_workspace_bytes(int64_t nv, int64_t nc, int n_out);
rbf_status rbf_deform_volume_fields(const double *d_xv, int64_t nv, const double *d_xb,
                                    const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                                    int n_out, const rbf_params *p, double *d_out, void *d_ws,
                                    size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * Modal volume deformation on the tensor cores: for k displacement fields
 * (modes) that share one support set, Eq. 6 for all of them is the product
 * D = Phi_vc W with W of size nc x n_out (n_out = 3 k, e.g. 96 for 32
 * modes).  Phi_vc is generated tile by tile in FP32, rounded to BF16 in
 * shared memory and multiplied on the tensor cores (tcgen05.mma, FP32
 * accumulation in tensor memory).
 *   mode RBF_MODAL_BF16   : one BF16 x BF16 product (BF16 rounding of phi and
 *                           W: relative errors of order 2^-9 per term).
 *   mode RBF_MODAL_BF16X3 : phi and W split into three BF16 parts each
 *                           (orders 1, 2^-9, 2^-18); the six products down
 *                           to order 2^-18 are accumulated (about FP32
 *                           accuracy).
 *   mode RBF_MODAL_F16X2  : phi and W split into two FP16 parts each (orders
 *                           1 and 2^-11; each column of W is first scaled by
 *                           a power of two into [-1, 1), undone on output);
 *                           the three products down to order 2^-11 x 2^-11
 *                           are accumulated.  Errors: about 2^-20 sum_j
 *                           |w_j phi_vj| plus 2^-24 sum_j |w_j| (phi below
 *                           the FP16 normal range, 6.1e-5, keeps an absolute
 *                           precision of 2^-25), with half the products of
 *                           BF16X3.
 * Errors against FP64 scale with sum_j |w_j phi_vj|, not with |D|: weights
 * of ill-conditioned support sets (large R) cancel heavily.
 *
 * d_w   : device FP64 nc x n_out (row-major, support order).
 * d_out : device FP32 nv x n_out (16-byte aligned).  n_out % 16 == 0,
 *         16 <= n_out <= 256, nc <= 4096 and the shared-memory tables must
 *         fit (RBF_E_ARG otherwise).
 * ASYNC; rbf_modal_check(d_ws) synchronises and returns the device status
 * (RBF_E_TIMEOUT if a bounded wait ran out).
 * ------------------------------------------------------------------------ */
#define RBF_MODAL_BF16 1
#define RBF_MODAL_F16X2 2
#define RBF_MODAL_BF16X3 3

size_t rbf_modal_workspace_bytes(int64_t nv, int64_t nc, int n_out, int mode);
rbf_status rbf_deform_modal(const double *d_xv, int64_t nv, const double *d_xb,
                            const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                            int n_out, const rbf_params *p, int mode, float *d_out,
                            void *d_ws, size_t ws_bytes, void *stream);
rbf_status rbf_modal_check(const void *d_ws, void *stream);

/* --------------------------------------------------------------------------
 * Batched volume sums (Eq. 6) for many problems in one double-float launch,
 * e.g. after rbf_greedy_batch_run.  The number of centres of each problem is
 * read on the device (d_nc, e.g. rbf_greedy_batch_nc_device(b) + i), so a
 * greedy batch and a volume batch can be captured together in one CUDA
 * graph.  The tile shape (threads per CTA, points per thread) is chosen at
 * create time by timing each candidate on the given problems -- create RUNS
 * the kernels (outputs are overwritten) and needs valid inputs, including
 * d_nc.  eval_prec must be RBF_PREC_F32X2; nc_max <= 1024.
 *   create: SYNCHRONOUS.  run: ASYNC (capturable).  info: chosen shape and
 *   the time of each candidate (4 floats, ms).
 * ------------------------------------------------------------------------ */
typedef struct {
    const double *d_xv;       /* device FP64 nv x 3 */
    int64_t nv;
    const double *d_xb;       /* device FP64 boundary coordinates */
    const int32_t *d_sel_idx; /* device int32[nc_max] */
    const double *d_w;        /* device FP64 nc_max x 3 */
    const int64_t *d_nc;      /* device: number of centres in use */
    int64_t nc_max;
    double radius;
    double *d_dv;             /* device FP64 nv x 3 (output) */
} rbf_volume_problem;

typedef struct rbf_volume_batch rbf_volume_batch;

size_t rbf_volume_batch_workspace_bytes(const rbf_volume_problem *h_probs, int B,
                                        int eval_prec);
rbf_status rbf_volume_batch_create(const rbf_volume_problem *h_probs, int B, int eval_prec,
                                   void *d_ws, size_t ws_bytes, void *stream,
                                   rbf_volume_batch **out);
rbf_status rbf_volume_batch_run(rbf_volume_batch *b, void *stream);
rbf_status rbf_volume_batch_info(const rbf_volume_batch *b, int *threads,
                                 int *points_per_thread, float *candidate_ms);
void rbf_volume_batch_destroy(rbf_volume_batch *b);

/* --------------------------------------------------------------------------
 * Volume displacements without any device allocation or caller workspace.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (for instance a plug-in whose host
 * application owns all device memory and forbids libraries from allocating,
 * or a time-critical loop that cannot afford an allocation's implicit
 * synchronisation) and therefore cannot hand rbf_deform_volume a workspace.
 * It computes the same FP32 sum as rbf_deform_volume with
 * eval_prec = RBF_PREC_F32, reading the volume points in place.
 *
 * Its scratch is a fixed array of RBF_NOALLOC_MAX_CENTRES (centre, weight)
 * entries (256 KiB) in device global memory, held on every device that has
 * used it until the process exits.  Under CUDA's default lazy module loading
 * the array is reserved when the driver loads the library's module on a
 * device, which happens inside the first call on that device: that call
 * looks up the array's device address (cudaGetSymbolAddress, with the device
 * current) and may synchronise the device.  Make the first call on each
 * device -- a call with nv = 0 counts, and does only this set-up -- outside
 * time-critical loops and before any stream capture.  Every call shares the
 * array and overwrites the entries it reads,
 * so results never depend on an earlier call, but calls whose GPU work
 * overlaps (different streams, or host threads) race on it: serialise them.
 * No cudaMalloc, cudaFree or other allocating routine is called.
 *
 * Arguments as rbf_deform_volume; p->eval_prec must be RBF_PREC_F32 and
 * nc <= RBF_NOALLOC_MAX_CENTRES, otherwise RBF_E_ARG.  ASYNC.
 * ------------------------------------------------------------------------ */
#define RBF_NOALLOC_MAX_CENTRES 8192

rbf_status rbf_deform_volume_noalloc(const double *d_xv, int64_t nv,
                                     const double *d_xb, const int32_t *d_sel_idx,
                                     int64_t nc, const double *d_w,
                                     const rbf_params *p, double *d_dv,
                                     void *stream);

/* --------------------------------------------------------------------------
 * Volume displacements (Eq. 6) with compact-support culling: the Wendland
 * C2 basis is zero for d >= R (Sec. 2), so pairs farther apart than R are
 * skipped.  A plan is made once per volume mesh, radius and precision: it
 * sorts the points along a Morton curve of a uniform cell grid and records
 * the bounding box of each tile of consecutive sorted points.  A run lists,
 * per tile and in support order, the centres within R (with a 1e-3 R
 * margin) of the tile's box and sums only those.  A skipped pair is an
 * exact zero of the unculled sum, so the result equals the unculled sum of
 * the same precision with its zero terms left out (bit for bit in
 * double-float; in FP32, pairs at d >= R are exact zeros here and
 * below 1e-28 of |w| in rbf_deform_volume).
 *
 * p->eval_prec: RBF_PREC_F32 or RBF_PREC_F32X2.  p->radius fixes the scaling
 * of the plan (every run uses it).  p->nc_max (>= 1): largest support set a
 * run may pass.  nv <= 2^31 - 1.
 * d_xv : device FP64 nv x 3, read by create only (the plan keeps its own
 *        packed, sorted copy in the workspace).
 * d_ws : device workspace of rbf_volume_plan_workspace_bytes(nv, p) bytes,
 *        256-byte aligned, owned by the caller and used by the plan until it
 *        is destroyed.
 * run  : d_xb, d_sel_idx, d_w as rbf_deform_volume (nc <= p->nc_max);
 *        d_dv device FP64 nv x 3 (output, original point order);
 *        d_pairs: NULL or a device counter to which the run adds the number
 *        of pairs it evaluated (the culled count is nv * nc minus it).
 * create: ASYNC (enqueued on `stream`, plan usable on that stream at once).
 * run: ASYNC (capturable).  info: plan shape (host).  destroy: host only.
 * ------------------------------------------------------------------------ */
typedef struct rbf_volume_plan rbf_volume_plan;

size_t rbf_volume_plan_workspace_bytes(int64_t nv, const rbf_params *p);
rbf_status rbf_volume_plan_create(const double *d_xv, int64_t nv, const rbf_params *p,
                                  void *d_ws, size_t ws_bytes, void *stream,
                                  rbf_volume_plan **out);
rbf_status rbf_volume_plan_run(const rbf_volume_plan *plan, const double *d_xb,
                               const int32_t *d_sel_idx, int64_t nc, const double *d_w,
                               double *d_dv, unsigned long long *d_pairs, void *stream);
rbf_status rbf_volume_plan_info(const rbf_volume_plan *plan, int *bits_per_axis,
                                int64_t *points_per_tile, int64_t *tiles);
void rbf_volume_plan_destroy(rbf_volume_plan *plan);

/* --------------------------------------------------------------------------
 * Kullback-Leibler divergence of two support sets (Sec. 4.1), the paper's
 * measure of how far a support-node distribution lies from another:
 *
 *     KL(S1 || S2) = sum_{i=1..N_b} d1_i log(d1_i / d2_i),
 *     dk_i = min over j in Sk of |r_i - r_j|   (Euclidean, FP64).
 *
 * Terms with d1_i = 0 or d2_i = 0 (node i belongs to a set) have no finite
 * logarithm and are left out (the paper is silent on them).
 * rbf_nearest_support: d_dist[i] = min over the nc listed nodes of
 * |r_i - r_j|, device FP64[nb] (output).  ASYNC.
 * rbf_support_kl: h_kl (host) = KL(S1 || S2); the sum is deterministic (a
 * fixed reduction tree).  SYNCHRONOUS.
 * d_xb: device FP64 nb x 3; d_sel*: device int32 node indices in [0, nb).
 * ------------------------------------------------------------------------ */
rbf_status rbf_nearest_support(const double *d_xb, int64_t nb, const int32_t *d_sel_idx,
                               int64_t nc, double *d_dist, void *stream);
size_t rbf_support_kl_workspace_bytes(int64_t nb);
rbf_status rbf_support_kl(const double *d_xb, int64_t nb, const int32_t *d_sel1, int64_t nc1,
                          const int32_t *d_sel2, int64_t nc2, double *h_kl, void *d_ws,
                          size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * The random partition rbf_greedy_select uses (Sec. 3: "stochastically and
 * uniformly" into m groups whose sizes differ by at most one), on the host:
 * h_group_of[node] = group of the node, 0..m-1.  SplitMix64(seed) drives a
 * Fisher-Yates shuffle (position i = nb-1 down to 1 swapped with
 * j = next() mod (i+1)); node perm[p] belongs to group p mod m.
 * HOST ONLY (no device needed).  Returns RBF_E_ARG for nb < 1, m < 1, m > nb.
 * ------------------------------------------------------------------------ */
rbf_status rbf_group_of(int64_t nb, int64_t m, uint64_t seed, int32_t *h_group_of);

/* --------------------------------------------------------------------------
 * Factorised support systems: Phi_SS X = B solved many times for one support
 * set (Sec. 2: Phi_SS is SPD and is solved through its Cholesky factor).
 * rbf_factor_create runs the recurrence-Cholesky appends once (as
 * rbf_solve_system does) and keeps Z = L^-1 in the workspace; each
 * rbf_factor_solve then costs X = Z^T Z B plus `refine_steps` FP64
 * refinement steps (residual recomputed from coordinates) instead of a new
 * factorisation.  d_xb and d_sel_idx must stay valid and unchanged while the
 * factor lives; the workspace (rbf_factor_workspace_bytes(nc), 256-byte
 * aligned) belongs to the factor until rbf_factor_destroy.
 * create: SYNCHRONOUS (RBF_E_NOT_SPD for coincident nodes).
 * solve: d_rhs, d_x device FP64 nc x 3 (support order); h_max_resid (host or
 * NULL) = max |Phi_SS X - B|_inf.  SYNCHRONOUS.  destroy: host only.
 * ------------------------------------------------------------------------ */
typedef struct rbf_factor rbf_factor;

size_t rbf_factor_workspace_bytes(int64_t nc);
rbf_status rbf_factor_create(const double *d_xb, int64_t nb, const int32_t *d_sel_idx,
                             int64_t nc, const rbf_params *p, void *d_ws, size_t ws_bytes,
                             void *stream, rbf_factor **out);
rbf_status rbf_factor_solve(const rbf_factor *f, const double *d_rhs, int refine_steps,
                            double *d_x, double *h_max_resid, void *stream);
void rbf_factor_destroy(rbf_factor *f);

/* --------------------------------------------------------------------------
 * Adjoint of the volume deformation for gradients with respect to the
 * support displacements d_c (Eq. 6 with Eqs. 4-5: d_v = Phi_vc W, Phi_cc W = d_c):
 *
 *     dJ/dd_c = Phi_cc^-1 Phi_vc^T dJ/dd_v      (Phi_cc symmetric)
 *
 * Phi_vc is recomputed pair by pair, never stored.  The transposed pair sum
 * runs in double-float (p->eval_prec = RBF_PREC_F32X2, recommended: the solve
 * amplifies right-hand-side errors by the condition number of Phi_cc) or
 * FP32 pairs, with FP64 accumulation across chunks of points and a fixed
 * (deterministic) reduction order; the solve is rbf_solve_system (FP64 with
 * p->refine_steps refinement steps).  The gradient with respect to all
 * boundary displacements is dJ/dd_c at the support nodes and 0 elsewhere.
 *
 * d_xv : device FP64 nv x 3;  d_gv : device FP64 nv x 3 (dJ/dd_v).
 * d_gc : device FP64 nc x 3 (output, support order).  nc <= 1024.
 * h_max_resid : host or NULL; residual of the final solve.
 * SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
size_t rbf_adjoint_workspace_bytes(int64_t nv, int64_t nc);

rbf_status rbf_deform_volume_adjoint(const double *d_xv, int64_t nv,
                                     const double *d_xb, int64_t nb,
                                     const int32_t *d_sel_idx, int64_t nc,
                                     const double *d_gv, const rbf_params *p,
                                     double *d_gc, double *h_max_resid,
                                     void *d_ws, size_t ws_bytes, void *stream);

/* The same with the support system already factorised (rbf_factor_create
 * on the same d_xb and support set): the solve reuses Z, so a gradient costs
 * the transposed pair sum and the refinement only.  p: eval_prec and
 * refine_steps are used (radius comes from the factor).  Workspace as
 * rbf_adjoint_workspace_bytes(nv, nc).  SYNCHRONOUS. */
rbf_status rbf_deform_volume_adjoint_factored(const double *d_xv, int64_t nv,
                                              const double *d_gv, const rbf_factor *f,
                                              const rbf_params *p, double *d_gc,
                                              double *h_max_resid, void *d_ws,
                                              size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------------
 * Vector-FMA peak microbenchmark of this GPU (dependent-FMA chains on every
 * SM), used as the denominator of the pair kernels' roofline.
 * prec: 32 (scalar FP32 FMA), 64 (FP64 FMA) or RBF_PEAK_F32X2 (paired FP32
 * FMA instructions, two FMAs each).  h_flops: host; measured FLOP/s (an FMA
 * counts 2).
 * SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
#define RBF_PEAK_F32X2 2
rbf_status rbf_measure_fma_peak(int prec, double *h_flops, void *stream);

/* --------------------------------------------------------------------------
 * Latency microbenchmarks: the parameters of the persistent greedy's cost
 * model, which is bound by latency rather than by a pipe or by memory.
 *   RBF_LAT_GRID_BARRIER: nanoseconds per grid barrier of the greedy kernels
 *     (the same barrier code) among `param` co-resident CTAs of 256 threads
 *     (RBF_E_ARG if they cannot all be resident);
 *   RBF_LAT_FP64_WARP / RBF_LAT_FP32_WARP: nanoseconds per FMA instruction
 *     of a lone warp running 8 independent chains (the issue cost one-warp
 *     scalar work pays).
 * h_ns: host, the best of two timed repetitions.  SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
#define RBF_LAT_GRID_BARRIER 1
#define RBF_LAT_FP64_WARP 2
#define RBF_LAT_FP32_WARP 3
rbf_status rbf_measure_latency(int what, int param, double *h_ns, void *stream);

/* --------------------------------------------------------------------------
 * Largest relative error of a hardware approximation over every normal
 * float x in [2^-126, 4), against the FP64 square root:
 *   RBF_APPROX_SQRT:  sqrt.approx.f32(x), used by the FP32 pair path;
 *   RBF_APPROX_RSQRT: rsqrtf(x) as compiled in this library, the start of
 *                     every double-float square root.
 * The certified error bounds of the screened evaluation (FP32 and
 * double-float modes of the greedy) assume at most 2^-22 for both; this
 * probe measures it on the device at hand.  h_max_rel: host.  No caller
 * memory is used (one library word in device memory).  SYNCHRONOUS.
 * ------------------------------------------------------------------------ */
#define RBF_APPROX_SQRT 1
#define RBF_APPROX_RSQRT 2
rbf_status rbf_measure_approx_error(int which, double *h_max_rel, void *stream);

/* Status latched by the last ASYNC call's device work on this device
 * (RBF_OK if none failed); reading it synchronises the device. */
rbf_status rbf_last_device_status(void);

/* Human-readable name of a status code (static storage). */
const char *rbf_status_string(rbf_status s);

/* Library version string (static storage). */
const char *rbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBFGCB_H */
