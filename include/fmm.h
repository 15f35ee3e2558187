/*
 * fmm.h -- C ABI of the GB300 balanced-tree fast multipole method.
 *
 * The method is the balanced-tree adaptive FMM of Bull & Engblom,
 * "Distributed and Adaptive Fast Multipole Method in Three Dimensions"
 * (arXiv:2002.04894): a tree of a fixed number of levels whose boxes are split
 * at median planes (Sec. 2.1.2, eta = 1; eta < 1 by option), theta-criterion connectivity
 * (Eq. 2.2), multipole/local expansions of order p (Sec. 2.1), and the stage
 * order of Algorithm 1 (Tree; P2M; M2M; M2L and L2L, Algorithm 3; L2P and P2P,
 * Algorithm 4). It evaluates, for N points x_i with real charges q_i,
 *
 *     phi_i = sum_{j != i} q_j / |x_i - x_j|                      (Eq. 2.1)
 *     E_i   = -grad phi_i = sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3
 *
 * with no physical constant. Pairs at zero distance contribute nothing.
 *
 * Conventions shared by every entry point:
 *  - A "level" is one binary bisection (median by default, see fmm_opts.eta):
 *    `levels` = B gives 2^B leaves
 *    and boxes numbered in heap order, box g = 2^l - 1 + j for box j of
 *    level l (children of g are 2g+1 and 2g+2).
 *  - Pointers to point, charge and output arrays may be device pointers or
 *    host pointers (pageable or pinned); the library detects which with
 *    cudaPointerGetAttributes and stages host data through device buffers.
 *    Device memory must belong to the current device (managed memory is
 *    accepted); a pointer into another GPU's memory is FMM_EINVAL.
 *    Host outputs are complete when the call returns; device work is
 *    asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).
 *  - All parity/inspection hooks (fmm_plan_tree, fmm_plan_list,
 *    fmm_eval_expansions, fmm_plan_stats) write HOST memory and synchronise
 *    the plan's stream.
 *  - Status codes are returned, never thrown; the library never aborts,
 *    traps or exits. Device-detected errors are reported by the call that
 *    next synchronises (fmm_plan always does).
 *  - Distinct plans may be used from distinct host threads concurrently; one
 *    plan must not be used by two threads at once.
 */
#ifndef FMM_H
#define FMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum fmm_status {
    FMM_OK = 0,
    FMM_EINVAL = -1,      /* bad argument: n < 1, levels or p out of range, theta not in [0,1),
                             unknown precision or flag bits */
    FMM_ENOMEM = -2,      /* the allocator returned NULL */
    FMM_ENONFINITE = -3,  /* a point coordinate is NaN or infinite */
    FMM_ECAPACITY = -4,   /* an interaction list exceeds 2^31 - 1 entries */
    FMM_ETIMEDOUT = -5,   /* a bounded device wait gave up (one-launch downward pass,
                             tensor-core M2L); reported by fmm_eval_check */
    FMM_ECUDA = -6,       /* a CUDA runtime call failed; fmm_last_cuda_error() has the code */
    FMM_EINTERNAL = -7    /* a device-side consistency check of the tree build failed (the
                             partition of a box did not give the sizes the split rule
                             requires); no CUDA error lies behind it */
};

/* Element type of points, charges and outputs. */
enum fmm_dtype { FMM_F64 = 0, FMM_F32 = 1 };

/*
 * Arithmetic of the evaluation stages.
 *  FMM_PREC_FP64  every stage in double precision (the plain form).
 *  FMM_PREC_MIXED box geometry, theta-test, M2M and L2L in double; P2M, M2L,
 *                 L2P and P2P in single precision with leaf-centred
 *                 coordinates and compensated per-target sums.
 */
enum fmm_prec { FMM_PREC_FP64 = 0, FMM_PREC_MIXED = 1 };

#define FMM_MAX_LEVELS 24
#define FMM_MAX_P 20

/* fmm_opts.flags bits */
#define FMM_FLAG_PROFILE 1  /* record per-stage device times (fmm_stage_times) */
#define FMM_FLAG_ETA 2      /* use fmm_opts.eta; without it eta = 1 (median splits) */
#define FMM_FLAG_TIGHT 8    /* box geometry from the points: the expansion centre and
                               radius of a box are the midpoint and half diagonal of
                               the bounding box of its own points (radius at least
                               2^-10 of the cell's; an empty box keeps its cell
                               midpoint) instead of its cell's. The cells still decide
                               the splits (fmm_plan_tree's lo/hi stay the cells).
                               Clustered inputs then get far fewer near-field pairs. */
#define FMM_FLAG_ROOT_CELL 16 /* the root cell is fmm_opts.root_lo/root_hi instead of the
                               points' bounding box. It must hold every point
                               (FMM_EINVAL otherwise). With it, the plan of the points
                               of one box of a larger tree, given in ascending original
                               index with that box's cell, is that box's subtree bit for
                               bit: how a rank builds its part of a tree split over
                               several devices. */
#define FMM_FLAG_TC_M2L 4   /* mixed form, p <= 12: M2L contractions on the tensor
                               cores (tcgen05, split TF32) instead of the CUDA cores;
                               same accuracy, slower at the orders measured (the
                               fixed matrices are at most 13 x 13) */

/* Stages of Algorithm 1 as timed by fmm_stage_times. */
enum fmm_stage {
    FMM_STAGE_TREE = 0,  /* fmm_plan: bounding box, median splits, cell geometry */
    FMM_STAGE_LISTS,     /* fmm_plan: theta-criterion connectivity */
    FMM_STAGE_P2M,       /* fmm_eval: charge gather + P2M */
    FMM_STAGE_M2M,
    FMM_STAGE_M2L,
    FMM_STAGE_L2L,
    FMM_STAGE_L2P,
    FMM_STAGE_P2P,       /* includes the scatter to input order */
    FMM_NSTAGES
};

typedef struct fmm_opts {
    int levels;     /* B: number of binary bisections, 0 <= B <= FMM_MAX_LEVELS */
    int p;          /* expansion order: degrees 0..p, 0 <= p <= FMM_MAX_P */
    double theta;   /* theta-criterion parameter (Eq. 2.2), 0 <= theta < 1;
                       theta = 0 gives no weak pairs (the FMM reduces to Eq. 2.1) */
    int prec;       /* enum fmm_prec */
    int flags;      /* FMM_FLAG_* bits; other bits must be 0 */
    double eta;     /* adaptivity of the splits (Sec. 2.1.2), 0 <= eta <= 1, read
                       only with FMM_FLAG_ETA. A box's cut plane is
                       eta * (median plane) + (1 - eta) * (cell midpoint) and the
                       lower child takes the points strictly below it: eta = 1 is
                       the balanced median split (equal halves), eta = 0 the
                       geometric bisection (children may be empty). For eta < 1
                       the build reads the largest child size back to the host
                       once per level. */
    int bisections_per_level;
                    /* bisections that make one expansion level: 0 or 1 (binary
                       levels, the default), 2, or 3 (the paper's octree levels,
                       8 children per box). `levels` counts bisections and must
                       be a multiple of it; connectivity (a parent pair yields
                       4^s candidate pairs), M2M, M2L and L2L then act only on
                       every s-th bisection level, and the levels between carry
                       empty lists and zero expansions. */
    double root_lo[3], root_hi[3];
                    /* root cell, read only with FMM_FLAG_ROOT_CELL (lo <= hi,
                       finite) */
} fmm_opts;

/*
 * Optional device allocator. alloc returns device memory of at least `bytes`
 * usable in stream order on `stream` (or NULL on failure); free releases it.
 * Without one the library allocates from a stream-ordered memory pool of its
 * own per device, which keeps freed memory for later plans instead of
 * returning it at every synchronisation; fmm_pool_trim releases it.
 */
typedef void *(*fmm_alloc_fn)(size_t bytes, void *ctx, void *stream);
typedef void (*fmm_free_fn)(void *ptr, size_t bytes, void *ctx, void *stream);
typedef struct fmm_allocator {
    fmm_alloc_fn alloc;
    fmm_free_fn free;
    void *ctx;
} fmm_allocator;

typedef struct fmm_plan_s *fmm_plan_t;

/*
 * fmm_plan -- build the balanced tree and its connectivity (Algorithm 2 on one
 * device; Sec. 2.1.1-2.1.2).
 *   points  n x 3 row-major coordinates, dtype `dtype`, host or device.
 *   n       number of points, 1 <= n <= 2^31 - 1.
 *   opts    levels, p, theta, precision, flags (copied).
 *   alloc   optional allocator (copied; must outlive the plan), or NULL.
 *   stream  cudaStream_t for all of the plan's device work.
 *   out     receives the plan handle (owned by the caller; fmm_destroy frees).
 * The root cell is the tight bounding box; each box is split on the longest
 * axis of its cell so that the left child holds the floor(n/2) smallest
 * (coordinate, original index) keys, at the plane halfway between the two
 * sides. The plan copies the points into leaf order and keeps no pointer to
 * `points`. Synchronises `stream` (it reads the list sizes).
 * Errors: FMM_EINVAL, FMM_ENONFINITE, FMM_ENOMEM, FMM_ECAPACITY,
 * FMM_EINTERNAL, FMM_ECUDA; on error *out is NULL and nothing is leaked.
 */
int fmm_plan(const void *points, int64_t n, int dtype, const fmm_opts *opts,
             const fmm_allocator *alloc, void *stream, fmm_plan_t *out);

/*
 * fmm_eval -- one FMM evaluation for the plan's points (Algorithm 1 after
 * Tree: P2M, M2M, M2L, L2L, L2P, P2P).
 *   charges     n charges, plan's dtype, host or device.
 *   potentials  n outputs phi_i, plan's dtype, input order, host or device.
 *   fields      n x 3 row-major outputs E_i = -grad phi_i, or NULL to skip.
 * Allocates nothing (all scratch belongs to the plan). Asynchronous on
 * `stream` when every pointer is device memory; otherwise it returns after
 * the host outputs are written.
 * Errors: FMM_EINVAL (NULL plan/charges/potentials), FMM_ECUDA.
 */
int fmm_eval(fmm_plan_t plan, const void *charges, void *potentials, void *fields,
             void *stream);

/* fmm_destroy -- release the plan and its device memory (stream-ordered on
 * the plan's stream). NULL is a no-op. */
void fmm_destroy(fmm_plan_t plan);

/*
 * fmm_direct -- the exact sum of Eq. 2.1 at selected targets, in double
 * precision on the device, for accuracy checks of fmm_eval.
 *   points, charges  n x 3 and n values (dtype), host or device.
 *   targets          ntargets int64 indices into [0, n), host or device.
 *   potentials       ntargets outputs (dtype); fields: ntargets x 3 or NULL.
 * Sources are summed in blocks with compensated (Neumaier) partial sums.
 * Allocates device staging only for host arguments (cudaMallocAsync).
 * Errors: FMM_EINVAL (n < 1, ntargets < 0, NULL pointers), FMM_ECUDA.
 */
int fmm_direct(const void *points, const void *charges, int64_t n, int dtype,
               const int64_t *targets, int64_t ntargets, void *potentials,
               void *fields, void *stream);

/* Plan statistics (host). Counts are exact, from the plan's lists. */
typedef struct fmm_stats {
    int64_t n, nbox, nleaf;
    int levels, p, prec, dtype;
    double theta;
    int64_t weak_pairs;          /* directed M2L pairs, all levels */
    int64_t strong_leaf_pairs;   /* directed P2P leaf pairs, self pairs included */
    int64_t p2p_interactions;    /* sum over strong leaf pairs of n_t * n_s */
    int64_t weak_pairs_level[FMM_MAX_LEVELS + 1];
    int64_t p2p_units;           /* near-field work units: a tile of a target leaf's points
                                    against a segment of its strong list */
    int64_t p2p_partial_slots;   /* partial sums of leaves whose strong list holds more than
                                    about 65536 source points and was cut into segments */
} fmm_stats;

/* fmm_plan_stats -- fill *out (synchronises the plan's stream for the
 * near-field pair count). Errors: FMM_EINVAL, FMM_ECUDA. */
int fmm_plan_stats(fmm_plan_t plan, fmm_stats *out);

/*
 * fmm_plan_tree -- copy the tree to host arrays (any may be NULL):
 *   perm    n     original index of the point in each leaf-order slot
 *   begin   nbox  first slot of each box;  count nbox  points per box
 *   lo, hi  nbox x 3 cell bounds;  centre nbox x 3;  radius nbox
 *   axis    nbox  split axis (longest cell axis; leaves too)
 *   plane   nbox  split coordinate (0 for leaves)
 * Errors: FMM_EINVAL, FMM_ECUDA.
 */
int fmm_plan_tree(fmm_plan_t plan, int64_t *perm, int64_t *begin, int64_t *count,
                  double *lo, double *hi, double *centre, double *radius,
                  int32_t *axis, double *plane);

/*
 * fmm_plan_list -- copy one connectivity list to host memory (Eq. 2.2).
 *   kind 0: weak (M2L) pairs of `level`;  kind 1: strong pairs of `level`
 *   (at level == levels, the P2P list). CSR over the 2^level target boxes of
 *   the level: ptr[2^level + 1] (int64), src[ptr[2^level]] (int32, box index
 *   within the level, ascending per target). Both orientations are stored.
 * If src is NULL only ptr is written (to size src). Errors: FMM_EINVAL, FMM_ECUDA.
 */
int fmm_plan_list(fmm_plan_t plan, int level, int kind, int64_t *ptr, int32_t *src);

/*
 * fmm_eval_expansions -- copy the multipole (which = 0) or local (which = 1)
 * coefficients left by the last fmm_eval to host memory: nbox x ncoef complex
 * values as (re, im) doubles, ncoef = (p+1)(p+2)/2, coefficient (n, m) with
 * 0 <= m <= n at n(n+1)/2 + m. Normalisation: M_n^m = sum_j q_j
 * conj(Y_n^m(x_j - c)), phi(c + s) = sum L_n^m conj(Y_n^m(s)), with
 * Y_n^m = (-1)^m r^n P_n^m(cos t) e^{i m phi} / (n+m)! (no Condon-Shortley phase)
 * and C_n^{-m} = (-1)^m conj(C_n^m). Multipoles of the levels above the first
 * level that has weak pairs are not formed (no stage reads them) and read as
 * zero; local expansions there are zero by definition. With
 * bisections_per_level = s > 1 the bisection levels that are not multiples of
 * s hold no expansions and read as zero too.
 * Errors: FMM_EINVAL, FMM_ECUDA.
 */
int fmm_eval_expansions(fmm_plan_t plan, int which, double *out);

/*
 * fmm_eval_check -- synchronise the plan's stream and report device-side
 * failures of the evaluations since the plan was built: FMM_ETIMEDOUT if a
 * bounded wait inside a kernel ran out (its results are then invalid),
 * FMM_OK otherwise. Errors: FMM_EINVAL, FMM_ECUDA.
 */
int fmm_eval_check(fmm_plan_t plan);

/*
 * fmm_stage_times -- device milliseconds of each stage (enum fmm_stage) of
 * the plan's construction (TREE, LISTS) and of its last fmm_eval (the rest),
 * measured with CUDA events on the plan's stream. Needs FMM_FLAG_PROFILE in
 * the plan's opts. Writes FMM_NSTAGES doubles to host memory; synchronises.
 * Errors: FMM_EINVAL (NULL, or profiling off), FMM_ECUDA.
 */
int fmm_stage_times(fmm_plan_t plan, double *ms);

/*
 * fmm_kernel_launches -- number of CUDA kernels this library has launched in
 * the process so far (all plans, all threads). For launch accounting.
 */
int64_t fmm_kernel_launches(void);

/*
 * fmm_orb_order_noalloc -- the leaf order of the balanced tree (the `perm`
 * that fmm_plan_tree reports for the same points and levels) for small point
 * sets, computed without allocating any device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- plug-ins inside a host application that
 * owns every byte of device memory and hands out only the buffers of a call,
 * and real-time loops whose latency budget has no room for an allocator call
 * (or its occasional synchronisation). It runs the same median-split kernels
 * as fmm_plan, with all of their scratch (both copies of the positions and
 * indices, the box cells, the selection state) in one static device array of
 * FMM_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   points  DEVICE pointer (current device), n x 3 row-major, dtype FMM_F64
 *           or FMM_F32.
 *   n       1 <= n <= FMM_NOALLOC_MAX_POINTS.
 *   levels  0 <= levels <= FMM_NOALLOC_MAX_LEVELS.
 *   perm    DEVICE pointer (current device), at least n int32: original
 *           index of each leaf-order slot.
 *   stream  cudaStream_t for the work.
 * The call enqueues the kernels and a device-to-device copy into perm on
 * `stream`, then copies the build's 4-byte status word to the host and
 * synchronises `stream`, so perm is complete when it returns FMM_OK.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current. Every call shares the one array and
 * re-initialises what must start cleared, so calls that overlap on the GPU
 * (other streams, other host threads) race and corrupt each other's results:
 * serialise them.
 * Errors: FMM_EINVAL (NULL pointers, host pointers or another device's
 * memory, n or levels out of range, bad dtype), FMM_ENONFINITE (a NaN or
 * infinite coordinate), FMM_EINTERNAL, FMM_ECUDA (fmm_last_cuda_error() has
 * the code).
 */
#define FMM_NOALLOC_MAX_POINTS 4096
#define FMM_NOALLOC_MAX_LEVELS 12
#define FMM_NOALLOC_SCRATCH_BYTES (1280u * 1024u)
int fmm_orb_order_noalloc(const void *points, int64_t n, int dtype, int levels, int32_t *perm,
                          void *stream);

/*
 * Batched evaluation of many independent systems (one graph launch).
 *
 * fmm_batch_create -- record the evaluation (fmm_eval) of nplans plans into
 * one CUDA graph. Plan i reads charges[i] and writes potentials[i] and
 * fields[i] (NULL entry: no field); all of these must be DEVICE pointers and
 * stay valid for the life of the batch. When every plan is mixed-precision
 * (FMM_PREC_MIXED) on binary levels with the single-precision M2L, and all
 * share the order p and the data type, the graph holds nine kernels that
 * each run one stage for every system at once (charges in / zeroing, P2M,
 * M2M, M2L, L2L, L2P, near field for 64- and 128-target tiles, partial-sum
 * combine); the systems' near-field work units are merged, heaviest first,
 * when the batch is made. Otherwise the plans' own evaluations are spread
 * over nstreams (1..64; 0 = 16) forked branches of the graph. `stream` is
 * the stream used for the set-up and the capture (a private one is made if
 * it is NULL). The plans must not be evaluated elsewhere while the batch
 * runs, and must outlive it. A wait of the batched downward pass that runs
 * out is reported by fmm_eval_check on that system's plan (FMM_ETIMEDOUT).
 * Errors: FMM_EINVAL, FMM_ENOMEM, FMM_ECUDA.
 * fmm_batch_launch -- run the recorded evaluations on `stream` (asynchronous).
 * fmm_batch_info -- the kernel launches one fmm_batch_launch makes, and
 * whether the batched stages (1) or per-plan branches (0) were recorded.
 * fmm_batch_destroy -- release the graph, its streams and tables (NULL: no-op).
 */
typedef struct fmm_batch_s *fmm_batch_t;
int fmm_batch_create(const fmm_plan_t *plans, int nplans, const void *const *charges,
                     void *const *potentials, void *const *fields, int nstreams, void *stream,
                     fmm_batch_t *out);
int fmm_batch_launch(fmm_batch_t batch, void *stream);
int fmm_batch_info(fmm_batch_t batch, int64_t *kernels, int *fused);
void fmm_batch_destroy(fmm_batch_t batch);

/*
 * One rank's part of a system split over several devices (Sec. 2.2 and
 * Algorithms 2-4: local trees under the ranks' boxes of the top levels,
 * halo lists between ranks, multipoles and leaf points exchanged for the
 * cross-rank M2L and P2P). The caller does the bookkeeping and the exchange
 * (paper_2002_04894_gb300/dist.py); these calls do the arithmetic. Plain FP64
 * plans only (FMM_EINVAL otherwise). All pointers are DEVICE memory of the
 * current device; work is asynchronous on `stream`. Boxes are given as
 * (level, index within the level) of the plan's own tree; coefficient arrays
 * are n x ncoef complex doubles, (n, m) at n(n+1)/2 + m as for
 * fmm_eval_expansions. Errors: FMM_EINVAL, FMM_ENOMEM, FMM_ECUDA.
 *
 * fmm_theta_test      weak[i] = 1 if boxes (ca[i], ra[i]) and (cb[i], rb[i])
 *                     are weakly connected by Eq. 2.2 (the list build's test,
 *                     bit for bit), else 0; centres n x 3.
 * fmm_eval_upward     charge gather, P2M and M2M on every level of the plan
 *                     (its root included); clears the received terms.
 * fmm_plan_multipoles out[i] = multipole of box idx[i] of `level`.
 * fmm_plan_add_locals adds L[i] to the local expansion of box idx[i].
 * fmm_m2l_external    adds the M2L of multipole M[i] about centre[i] to the
 *                     local expansion of box tgt[i] of `level`.
 * fmm_plan_leaf_points the points of leaves leaf[i] as (x, y, z, q) doubles
 *                     from row off[i] of out (off: n + 1 int64, the caller's
 *                     prefix sum of the leaves' counts from fmm_plan_tree).
 * fmm_p2p_external    adds to the points of leaf tgt[i] the potential and
 *                     field of the sources src[off[i] .. off[i+1]) (x, y, z, q
 *                     rows; pairs at zero distance skipped).
 * fmm_eval_downward   M2L within the plan, the added local expansions, L2L,
 *                     L2P, the received near-field terms and P2P: potentials
 *                     and fields in the order the plan's points were given.
 * fmm_translate       for i < n, dst[i] += the translation of src[i] about
 *                     csrc[i] to cdst[i]: kind 0 M2M, 1 M2L, 2 L2L (direct
 *                     sums; for the few boxes above the ranks' subtrees).
 */
int fmm_theta_test(double theta, int64_t n, const double *ca, const double *ra, const double *cb,
                   const double *rb, uint8_t *weak, void *stream);
int fmm_eval_upward(fmm_plan_t plan, const void *charges, void *stream);
int fmm_plan_multipoles(fmm_plan_t plan, int level, int64_t n, const int32_t *idx, double *out, void *stream);
int fmm_plan_add_locals(fmm_plan_t plan, int level, int64_t n, const int32_t *idx, const double *L,
                        void *stream);
int fmm_m2l_external(fmm_plan_t plan, int level, int64_t n, const int32_t *tgt, const double *M,
                     const double *centre, void *stream);
int fmm_plan_leaf_points(fmm_plan_t plan, int64_t n, const int32_t *leaf, const int64_t *off, double *out,
                         void *stream);
int fmm_p2p_external(fmm_plan_t plan, int64_t n, const int32_t *tgt, const int64_t *off, const double *src,
                     void *stream);
int fmm_eval_downward(fmm_plan_t plan, void *potentials, void *fields, void *stream);
int fmm_translate(int kind, int p, int64_t n, const double *src, const double *csrc, const double *cdst,
                  double *dst, void *stream);

/*
 * fmm_measure_peak -- throughput of one arithmetic pipe of the current device,
 * the denominator of the evaluation kernels' rooflines (not part of the
 * method). kind: 0 FP32 FFMA, 1 FP32 packed FFMA2, 2 FP64 DFMA (flop/s, two
 * per multiply-add), 3 XU rsqrt.approx (operations/s). Independent chains of
 * that instruction on 4 blocks of 256 threads per SM, `iters` iterations per
 * thread (32 flop per iteration for kinds 0 and 1, 16 for 2, 8 rsqrt for 3),
 * timed with CUDA events on `stream` after one untimed launch of iters/8.
 * Writes the rate to *ops_per_s and the timed launch's milliseconds to *ms
 * (may be NULL); synchronises `stream`. Allocates nothing.
 * Errors: FMM_EINVAL (NULL output, iters < 1, unknown kind), FMM_ECUDA.
 */
int fmm_measure_peak(int kind, int64_t iters, void *stream, double *ops_per_s, double *ms);

/*
 * fmm_set_list_capacity -- set the largest number of candidate pairs one
 * level of the connectivity build may hold (default and maximum 2^31 - 1,
 * the int32 index range of the lists); returns the previous value. A value
 * outside 1 .. 2^31 - 1 restores the default. Process-wide. It exists so
 * that tests can make fmm_plan meet FMM_ECAPACITY on small inputs; plans
 * already built are not affected.
 */
int64_t fmm_set_list_capacity(int64_t entries);

/*
 * fmm_set_wait_limit -- the bound of the device-side waits of the one-launch
 * downward pass (a box waits for its parent's expansion): `sleeps` waits of
 * ~0.1 us each before the wait gives up and the evaluation reports
 * FMM_ETIMEDOUT through fmm_eval_check (default and any value <= 0: 2^24,
 * ~2 s). `withhold` > 0 names a box (heap index) whose completion is never
 * signalled, so that its children's waits run out: a test of the timeout
 * path that needs no device fault (<= 0: none). Process-wide; returns the
 * previous limit.
 */
int64_t fmm_set_wait_limit(int64_t sleeps, int64_t withhold);

/* fmm_strerror -- static text for a status code. */
const char *fmm_strerror(int status);

/* fmm_last_cuda_error -- the cudaError_t behind the calling thread's last FMM_ECUDA. */
int fmm_last_cuda_error(void);

/*
 * fmm_pool_trim -- return the memory cached by the library's own pool on CUDA
 * device `device` (plans made without an allocator) to the system; memory
 * of live plans stays. A device whose pool was never used: FMM_OK.
 * Errors: FMM_EINVAL (device outside 0..63), FMM_ECUDA.
 */
int fmm_pool_trim(int device);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H */
