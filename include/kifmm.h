/*
 * kifmm.h -- C ABI of the GB300 Laplace kernel-independent FMM.
 *
 * The library evaluates the 3D Laplace N-body sum, Eq. (1) of "The Fast
 * Multipole Method" section:
 *
 *     phi_j = sum_{i != j} q_i / (4 pi |x_i - x_j|),   j = 1..n,
 *
 * with the kernel-independent FMM the paper implements: a linear octree split
 * while a box holds more than ncrit points, the U/V/W/X interaction lists
 * ("Computational structure of FMM operators": near field, M2L, M2P, P2L),
 * check and equivalent surfaces of 6(p-1)^2 + 2 points, and the operators
 * P2M, M2M, M2L, L2L, P2L, L2P, M2P and the near field (P2P).
 *
 * All types are plain C; no PyTorch or CUDA runtime type appears in a
 * signature.  A cudaStream_t is passed as void*.
 *
 * Errors: every entry point returns an fmm_status and never aborts the
 * process.  fmm_last_error() returns a thread-local message for the last
 * failure on the calling thread.
 */
#ifndef KIFMM_H
#define KIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan_s *fmm_plan_t; /* opaque, owned by the library */

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID_ARG = 1, /* bad pointer, size, option or state */
    FMM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    FMM_ERR_OOM = 3,         /* host or device allocation failed */
    FMM_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    FMM_ERR_UNSUPPORTED = 5  /* valid request this build does not handle */
} fmm_status;

/* Arithmetic used for the V-list M2L translations. */
typedef enum {
    FMM_M2L_FP32 = 0,   /* FP32 FMA on the CUDA cores */
    FMM_M2L_BF16X3 = 1, /* tcgen05 kind::f16, hi/lo BF16 split, 3 products */
    FMM_M2L_TF32X3 = 2  /* tcgen05 kind::tf32, hi/lo TF32 split, 3 products */
} fmm_m2l_mode;

/* Where a plan's octree, point order and U/V/W/X lists are built.  Every
   choice gives the same arrays, bit for bit. */
typedef enum {
    FMM_TREE_AUTO = 0,        /* on the device for a problem of at least
                                 65536 points (unless host_only), else
                                 FMM_TREE_HOST */
    FMM_TREE_HOST = 1,        /* recursive splitting and a balance worklist
                                 on the host */
    FMM_TREE_DEVICE = 2,      /* level-synchronous passes on the plan's CUDA
                                 device: Morton radix sort, split sets per
                                 level, balance from the deepest level up,
                                 lists by per-box neighbour lookups;
                                 positions may be host or device pointers */
    FMM_TREE_LEVELS_HOST = 3  /* the same level-synchronous passes in host
                                 loops (OpenMP) */
} fmm_tree_build;

/* Plan options.  fmm_options_init() fills the defaults given here. */
typedef struct {
    double alpha_inner; /* radius of upward-equivalent / downward-check
                           surfaces in box half-widths (1.05) */
    double alpha_outer; /* radius of upward-check / downward-equivalent
                           surfaces (2.95); must be < 3 */
    double rcond;       /* pseudo-inverse cutoff: singular values below
                           rcond * sigma_max are dropped (1e-7) */
    double eps_svd;     /* M2L compression: rank k = number of singular
                           values of the stacked M2L operators above
                           eps_svd * sigma_max; 0 keeps them dense (1e-7) */
    int32_t max_level;  /* deepest octree level, <= 16 (16) */
    int32_t balance;    /* 1: refine to the 2:1 balance condition (1) */
    int32_t m2l_mode;   /* fmm_m2l_mode (FMM_M2L_FP32) */
    int32_t host_only;  /* 1: build tree, lists and operators on the host
                           only; fmm_evaluate then returns
                           FMM_ERR_INVALID_ARG.  For inspection. (0) */
    int32_t device;     /* CUDA device ordinal; -1 = current device (-1) */
    int32_t tree_build; /* fmm_tree_build: where the octree and the lists
                           are built (FMM_TREE_AUTO) */
    int32_t direct_wx;  /* 1: a W-list box with no more points than a
                           surface (6(p-1)^2+2) acts on the leaf's points
                           through its points instead of its upward
                           equivalent surface (M2P), and a leaf with no
                           more points than a surface takes its X list's
                           points directly instead of through its downward
                           check surface (P2L); exact, and fewer pairs.
                           0: M2P and P2L for every W and X entry (1) */
    int32_t reserved[5];
} fmm_options;

void fmm_options_init(fmm_options *opts);

/*
 * On-disk cache of the FP64 operator precomputation (surfaces, factored
 * pseudo-inverses, M2M/L2L, the compressed M2L factors), which depends only
 * on (p, alpha_inner, alpha_outer, rcond, eps_svd) and takes seconds at
 * p >= 6.  The paper likewise precomputes the M2M and L2L matrices once
 * ("Parallelization strategies for FMM operators") and keeps trees and
 * precomputed quantities in a database ("Data-oriented design of
 * PyExaFMM").
 *
 * dir      an existing directory, or NULL / "" to turn the cache off (the
 *          default).  Process-wide; affects plans created afterwards.
 *
 * With a directory set, a plan whose operators are not yet in this
 * process's memory reads them from dir (one file per key, named
 * kifmm_ops_v<format>_p<p>_<hash of the radii and cutoffs>.bin) and, when
 * the file is missing or fails a check (key compared bit for bit, sizes,
 * checksum), computes them and writes the file through a temporary file
 * renamed into place.  Operators read from a file are bit-identical to the
 * ones written.  Failing to write is not an error.  Returns
 * FMM_ERR_INVALID_ARG if dir is not an existing directory.
 */
fmm_status fmm_set_operator_cache(const char *dir);

/*
 * Build a plan: octree, interaction lists, FP64 operator precomputation and
 * the device copies the evaluation needs.
 *
 * sources  n x 3 row-major FP64 positions, host or device pointer (detected).
 * targets  NULL or equal to sources: the targets are the sources, as in
 *          Eq. (1), and a pair at distance 0 (the point itself, or a
 *          coincident duplicate) is skipped.  Otherwise n x 3 FP64 target
 *          positions (host or device): the tree is built on the union of
 *          the 2n points, targets carry no charge, and the potential at
 *          each target sums every source at a non-zero distance.
 * n        number of sources (and of targets), >= 1.
 * p        expansion order, 2 <= p <= 10 (surface points 6(p-1)^2 + 2).
 * ncrit    largest number of points in a leaf before it is split, >= 1.
 * out      receives the plan; untouched on failure.
 *
 * The plan copies what it needs; the caller keeps ownership of every
 * pointer.  Synchronous with respect to the host.
 */
fmm_status fmm_plan_create(const double *sources, const double *targets,
                           int64_t n, int p, int ncrit, fmm_plan_t *out);

/* As fmm_plan_create, with options (NULL = defaults). */
fmm_status fmm_plan_create_ex(const double *sources, const double *targets,
                              int64_t n, int p, int ncrit,
                              const fmm_options *opts, fmm_plan_t *out);

/*
 * Build one plan for `nproblems` independent problems (batched evaluation).
 * The paper states one problem, Eq. (1); evaluating many of uneven size in
 * the same launches is this library's batching form of it.  Problem i has
 * n[i] >= 1 sources at sources[i] (n[i] x 3 FP64, host or device) and
 * targets[i] (NULL, or NULL array, or equal to sources[i]: the sources
 * themselves; else n[i] x 3 FP64 targets, as in fmm_plan_create).  The
 * problems share nothing but the launches: each has its own root cube,
 * octree and lists, and no interaction crosses problems.
 *
 * fmm_evaluate on such a plan takes charges of sum(n) x nrhs rows, problem
 * 0's rows first, and writes potentials in the same row order.
 * 1 <= nproblems <= 65536; sum(n) obeys the limit of fmm_plan_create.
 */
fmm_status fmm_plan_create_batch(const double *const *sources, const double *const *targets,
                                 const int64_t *n, int nproblems, int p, int ncrit,
                                 fmm_plan_t *out);
/* As fmm_plan_create_batch, with options (NULL = defaults). */
fmm_status fmm_plan_create_batch_ex(const double *const *sources,
                                    const double *const *targets, const int64_t *n,
                                    int nproblems, int p, int ncrit,
                                    const fmm_options *opts, fmm_plan_t *out);

/* Evaluation-time options that may change after creation. */
enum {
    FMM_OPT_M2L_MODE = 1, /* value: an fmm_m2l_mode */
    FMM_OPT_AUTOTUNE = 3, /* value 1 (default): the first evaluation of each
                             nrhs times every tile shape of each level
                             product (the batched matrix products of the
                             upward and downward passes) and keeps the
                             fastest; later evaluations use those.  The
                             shapes give bit-identical results.  0: the
                             default shape everywhere. */
    FMM_OPT_GEMM_SHAPE = 4,/* value -1 (default): shapes as the autotuner
                             (or its default) chooses; 0 .. 4: that shape
                             (64x32, 32x64, 128x16 with 4x4 tiles per
                             thread, 64x64, 128x32 with 8x4 tiles; rows x
                             vectors) for every level product. */
    FMM_OPT_GRAPH = 2,    /* value 1 (default): fmm_evaluate captures its
                             kernels into a CUDA graph on the first call for
                             a given (charges, potentials, nrhs, M2L mode)
                             and replays the graph on later calls with the
                             same ones; 0: launch the kernels directly.  The
                             legacy default stream (NULL) always launches
                             directly, since it cannot be captured. */
    FMM_OPT_TEST_M2L_STALL = 5, /* failure-detection test hook, value 0
                             (default) or 1.  With 1, block 0 of every
                             tensor-core M2L launch first waits on a barrier
                             that nothing completes; the wait gives up after
                             0.1 s, the block sets the plan's error word and
                             abandons its tiles (the other blocks finish), so
                             the evaluation's results are invalid and the
                             next call that checks the word (the same call
                             with host buffers, else the next evaluation)
                             returns FMM_ERR_TIMEOUT, roles mask 32.  The
                             plan stays usable.  No effect in FP32 mode. */
    FMM_OPT_M2L_KERNEL = 6,/* which tensor-core M2L kernel the BF16x3 and
                             TF32x3 modes run: 0 the pair-column kernel
                             (each V pair one column of a product by S_t,
                             in windows of up to 256 target boxes; needs an
                             operand width kpad <= 128, else the target-tile
                             kernel runs), 1 (default) the target-tile
                             kernel (128 target boxes of one level and
                             parity class per product).  Both sum each
                             target's offsets in the same order: the
                             results agree to rounding. */
    FMM_OPT_FORCE_KNOBS = 7 /* value -1 (default): the autotuner (first
                             evaluation of each nrhs) also times two
                             choices that change no result and keeps the
                             faster: the target-tile M2L's block schedule
                             and the leaf pass's launch order (see
                             FMM_ARRAY_TUNED_KNOBS); 0..3 sets them instead:
                             bit 0 = longest-first M2L tile schedule (else
                             round robin), bit 1 = leaf width groups
                             narrowest first (else widest first). */
};
fmm_status fmm_plan_set_option(fmm_plan_t plan, int key, double value);

/*
 * Evaluate potentials, Eq. (1), for nrhs charge vectors at once.
 *
 * charges     n x nrhs row-major FP32, in the caller's point order.
 * nrhs        >= 1.
 * potentials  n x nrhs row-major FP64, overwritten, caller's point order.
 * stream      cudaStream_t (NULL = legacy default stream).
 *
 * If charges and potentials are both device pointers the call only enqueues
 * work on `stream` and returns.  If either is a host pointer the library
 * stages it through device memory on `stream` and returns after the stream
 * has finished the evaluation.  A plan is not reentrant: do not overlap two
 * evaluations of one plan.  Device-side failures are reported by the next
 * call that synchronises.
 */
fmm_status fmm_evaluate(fmm_plan_t plan, const float *charges, int nrhs,
                        double *potentials, void *stream);

/*
 * Gradients of the potentials with respect to the target positions (the
 * field is minus this), beside or instead of the potentials:
 *
 *     grad_j = sum_{i != j} q_i (x_i - y_j) / (4 pi |x_i - y_j|^3),
 *
 * the derivative of Eq. (1) in the target position.  The kernel-independent
 * method admits it ("The Fast Multipole Method" section: any kernel the
 * evaluation step can apply): the upward and downward passes and the M2L are
 * those of fmm_evaluate; only the leaf step (near field over U, L2P, M2P)
 * applies the target-gradient of the kernel, in FP32 with Kahan-compensated
 * sums and the same close-pair correction, then FP64 output.
 *
 * gradients   n x nrhs x 3 row-major FP64, overwritten, caller's point order.
 * potentials  as in fmm_evaluate, or NULL (not written).
 * charges, stream, host/device pointers and synchronisation: as in
 * fmm_evaluate.  NULL gradients return FMM_ERR_INVALID_ARG.
 */
fmm_status fmm_evaluate_gradient(fmm_plan_t plan, const float *charges, int nrhs,
                                 double *potentials, double *gradients, void *stream);

/*
 * The evaluation of fmm_evaluate without any device allocation.  The paper
 * has no counterpart: this serves callers that may not allocate device
 * memory while they evaluate -- an application whose device memory is owned
 * by another allocator, a latency-critical loop in which cudaMalloc/cudaFree
 * would add their implicit device-wide synchronisation, or a service that
 * must not grow its device footprint after start-up.  (fmm_evaluate
 * allocates its workspace on its first call and whenever nrhs grows.)
 *
 * The workspace comes from one fixed 64 MiB array in device memory that the
 * library holds on every GPU that loads it, until the process exits.  The
 * first call on a device looks the array up (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  A reset
 * of the device's primary context (cudaDeviceReset) gives the array a new
 * address: the next call notices and looks it up again, so after a reset
 * that next call, too, should come before any stream capture.  The calling
 * thread's current device is the same on return as on entry.
 *
 * charges, potentials: device pointers only, layouts as in fmm_evaluate;
 * host pointers return FMM_ERR_INVALID_ARG.  A plan and nrhs whose workspace
 * exceeds 64 MiB return FMM_ERR_INVALID_ARG with the sizes in the message.
 * Every call on a device shares the array and overwrites it; nothing in it
 * has to start at zero.  Calls whose work overlaps on the GPU (different
 * streams, or different plans, on one device) race on the array: order them
 * on one stream or synchronise between them.
 */
fmm_status fmm_evaluate_noalloc(fmm_plan_t plan, const float *charges, int nrhs,
                                double *potentials, void *stream);

/* Destroy a plan and free its host and device memory.  NULL is a no-op. */
void fmm_destroy(fmm_plan_t plan);

/* Thread-local message describing the last failure on this thread. */
const char *fmm_last_error(void);

/* ---------------------------------------------------------------------
 * Inspection (host data of a plan; used by tests and tools)
 * ------------------------------------------------------------------- */

/* Integer facts about a plan. */
enum {
    FMM_INFO_N = 0,           /* rows of charges / potentials (sum of n) */
    FMM_INFO_NODES = 1,       /* boxes that hold points */
    FMM_INFO_LEAVES = 2,      /* leaves that hold points */
    FMM_INFO_DEPTH = 3,       /* deepest level */
    FMM_INFO_NSURF = 4,       /* surface points per box, 6(p-1)^2 + 2 */
    FMM_INFO_RANK_M2L = 5,    /* compressed M2L rank k */
    FMM_INFO_RANK_UP = 6,     /* kept singular values of the upward
                                 check-to-equivalent matrix */
    FMM_INFO_RANK_DOWN = 7,   /* same, downward */
    FMM_INFO_U_PAIRS = 8,     /* sum over leaves of |U| */
    FMM_INFO_V_PAIRS = 9,     /* sum over boxes of |V| */
    FMM_INFO_W_PAIRS = 10,    /* sum over leaves of |W| */
    FMM_INFO_X_PAIRS = 11,    /* sum over boxes of |X| */
    FMM_INFO_P2P_PAIRS = 12,  /* near-field (target, source) pairs */
    FMM_INFO_M2L_TILES = 13,  /* M2L target tiles */
    FMM_INFO_M2L_ENTRIES = 14,/* M2L (tile, offset) entries */
    FMM_INFO_LAST_LAUNCHES = 15,/* kernels the last evaluation launched */
    FMM_INFO_POINTS = 16,     /* points in the tree (2n with distinct
                                 targets) */
    FMM_INFO_PROBLEMS = 17,   /* independent problems */
    FMM_INFO_M2L_WINDOWS = 20,/* pair-column M2L windows */
    FMM_INFO_M2L_ITEMS = 21,  /* pair-column M2L items (offset products) */
    FMM_INFO_M2L_KERNEL = 22, /* M2L kernel of the current mode: 0 FP32 SIMT,
                                 1 tensor-core target tiles, 2 tensor-core
                                 pair columns */
    FMM_INFO_TUNINGS = 23,    /* autotuning evaluations so far (one per nrhs;
                                 the choices are kept per nrhs) */
    FMM_INFO_SURF_PAIRS = 24, /* leaf-pass (point, surface point) pairs:
                                 L2P from the leaf's own downward equivalent
                                 surface (levels >= 2) and M2P from the
                                 upward equivalent surface of every W box
                                 not taken directly (see direct_wx) */
    FMM_INFO_WX_DIRECT_PAIRS = 25, /* leaf-pass (point, point) pairs from W
                                 boxes and X leaves taken directly */
    FMM_INFO_OPERATOR_SOURCE = 19, /* where the plan's operators came
                                 from: 0 computed, 1 this process's memory,
                                 2 the operator cache file */
    FMM_INFO_DEVICE_TREES = 18 /* problems whose octree and lists were built
                                 on the device */
};
fmm_status fmm_plan_info(fmm_plan_t plan, int key, int64_t *value);

/* Arrays a plan can export.  Sizes are in elements of the stated type. */
enum {
    FMM_ARRAY_NODE_KEYS = 0, /* int32 [nodes][4]: level, ix, iy, iz, in
                                plan order (level, then problem, then
                                Morton order) */
    FMM_ARRAY_NODE_RANGE = 1,/* int64 [nodes][2]: first, end point index in
                                the sorted order */
    FMM_ARRAY_LEAF_FLAG = 2, /* int32 [nodes] */
    FMM_ARRAY_PERM = 3,      /* int64 [points]: sorted position -> input
                                point (sources, then targets if distinct;
                                problems concatenated) */
    FMM_ARRAY_U_PTR = 4,     /* int64 [nodes+1]: CSR offsets of U lists */
    FMM_ARRAY_U_IDX = 5,     /* int32 [U pairs]: node indices */
    FMM_ARRAY_V_PTR = 6,
    FMM_ARRAY_V_IDX = 7,
    FMM_ARRAY_W_PTR = 8,
    FMM_ARRAY_W_IDX = 9,
    FMM_ARRAY_X_PTR = 10,
    FMM_ARRAY_X_IDX = 11,
    FMM_ARRAY_SURFACE = 12,  /* double [nsurf][3] unit surface points */
    FMM_ARRAY_M2L_U = 13,    /* double [nsurf][k]: left factor U_k */
    FMM_ARRAY_M2L_V = 14,    /* double [nsurf][k]: right factor V_k */
    FMM_ARRAY_M2L_S = 15,    /* double [316][k][k]: S_t = U_k^T K_t V_k,
                                offsets t in lexicographic (tx,ty,tz) order
                                over {-3..3}^3 minus {-1..1}^3 */
    FMM_ARRAY_ROOT = 16,     /* double [problems][4]: root centre x, y, z,
                                half-width */
    FMM_ARRAY_CHARGE_ROW = 17,/* int64 [points]: charge row of each sorted
                                point, -1 for a target only */
    FMM_ARRAY_OUTPUT_ROW = 18,/* int64 [points]: potential row of each sorted
                                point, -1 for a source only */
    FMM_ARRAY_NODE_PROBLEM = 19,/* int32 [nodes]: problem of each box */
    FMM_ARRAY_GEMM_SHAPES = 20,/* int32 [level products]: the tile shape the
                                autotuner chose for each, in evaluation order
                                (empty before the first tuned evaluation) */
    /* The M2L work table ("M2L" of "Computational structure of FMM
     * operators": every target box B sums the translated densities of its
     * V list).  Targets with a non-empty V list are grouped per level and
     * per parity class (ix&1, iy&1, iz&1), in plan order, into tiles of 128
     * rows; an entry is one (tile, offset t) pair with the V-list source of
     * every row that has one at offset t. */
    FMM_ARRAY_M2L_TILE_LEVEL = 21,    /* int32 [tiles]: level of the tile */
    FMM_ARRAY_M2L_TILE_TARGET = 22,   /* int32 [tiles][128]: target box of
                                         each row, -1 past the last */
    FMM_ARRAY_M2L_TILE_ENTRY_PTR = 23,/* int32 [tiles+1]: CSR offsets of the
                                         tiles' entries */
    FMM_ARRAY_M2L_ENTRY_OFFSET = 24,  /* int32 [entries]: offset index t in
                                         the order of FMM_ARRAY_M2L_S,
                                         increasing within a tile */
    FMM_ARRAY_M2L_ENTRY_SRC = 25,     /* int32 [entries][128]: source box of
                                         each row at that offset, -1 none */
    /* FP64 operators of the unit box (half-width 1, kernel 1/r): the
     * matrices behind P2M, M2M, L2L and M2L ("Computational structure of
     * FMM operators": bottom-up M2M, top-down M2L and L2L), row-major;
     * rP = FMM_INFO_RANK_UP, rQ = FMM_INFO_RANK_DOWN, k = FMM_INFO_RANK_M2L,
     * s the unit surface, c_sigma = ((sigma&1) - 1/2, (sigma>>1&1) - 1/2,
     * (sigma>>2&1) - 1/2) the centre of child sigma. */
    FMM_ARRAY_OP_PU = 26,  /* double [nsurf][rP]: K(a_out s, a_in s) = */
    FMM_ARRAY_OP_PS = 27,  /* double [rP]:          Pu diag(Ps) Pv^T,   */
    FMM_ARRAY_OP_PV = 28,  /* double [nsurf][rP]:   truncated SVD       */
    FMM_ARRAY_OP_QU = 29,  /* double [nsurf][rQ]: K(a_in s, a_out s) = */
    FMM_ARRAY_OP_QS = 30,  /* double [rQ]:          Qu diag(Qs) Qv^T    */
    FMM_ARRAY_OP_QV = 31,  /* double [nsurf][rQ] */
    FMM_ARRAY_OP_M2M = 32, /* double [8][rP][nsurf]: Pu^T K(a_out s,
                              c_sigma + a_in s / 2) */
    FMM_ARRAY_OP_L2L = 33, /* double [8][rQ][nsurf]: Qu^T K(c_sigma +
                              a_in s / 2, a_out s) / 2 */
    FMM_ARRAY_OP_QUK = 34, /* double [rQ][k]: Qu^T Uk */
    /* the pair-column M2L work table (all int32): windows of target boxes
     * (boxes with a V list, in plan order), per window its items (one
     * offset each, in increasing offset order, at most 128 pairs), per item
     * its pairs (source box, target's place in the window), and the
     * windows each persistent block takes */
    FMM_ARRAY_M2L_WIN_TARGET_PTR = 35, /* [windows+1] */
    FMM_ARRAY_M2L_WIN_TARGETS = 36,    /* [V targets] */
    FMM_ARRAY_M2L_WIN_ITEM_PTR = 37,   /* [windows+1] */
    FMM_ARRAY_M2L_ITEM_OFFSET = 38,    /* [items]: offset index */
    FMM_ARRAY_M2L_ITEM_PAIR_PTR = 39,  /* [items+1] */
    FMM_ARRAY_M2L_PAIR_SRC = 40,       /* [V pairs]: source box */
    FMM_ARRAY_M2L_PAIR_SLOT = 41,      /* [V pairs]: target's place in its window */
    FMM_ARRAY_M2L_CTA_PTR = 42,        /* [blocks+1] */
    FMM_ARRAY_M2L_CTA_WIN = 43,        /* [windows]: window ids per block */
    /* the target-tile M2L's block schedule (int32; empty when the plan has
     * fewer tiles than the device has SMs): tiles dealt longest first
     * (cost = entries) to the least loaded persistent block */
    FMM_ARRAY_M2L_TILE_CTA_PTR = 44,   /* [blocks+1] */
    FMM_ARRAY_M2L_TILE_CTA_TILES = 45, /* [tiles]: tile ids per block */
    FMM_ARRAY_TUNED_KNOBS = 46         /* int32 [2]: the choices of the last
                                          evaluation: the M2L block schedule
                                          (1 longest-first tiles, 0 round
                                          robin) and the leaf pass's launch
                                          order (0 widest first, 1 narrowest
                                          first) */
};
/* Copy array `which` into dst (capacity `bytes`).  *needed receives the
 * size in bytes (may be NULL).  dst == NULL only queries the size. */
fmm_status fmm_plan_get_array(fmm_plan_t plan, int which, void *dst,
                              int64_t bytes, int64_t *needed);

/* Per-box results of the passes of the last fmm_evaluate (or
 * fmm_evaluate_gradient) on this plan, for per-operator tests: FP32
 * [nodes][nrhs][ld] in plan node order (FMM_ARRAY_NODE_KEYS), nrhs of that
 * evaluation.  Unit-box convention: in box B's coordinates y' = (y - c_B) / h_B
 * (h_B its half-width) the arrays stand for the potential
 *     phi(y) = sum_j rho_j / |y' - a s_j|  /  (4 pi h_B)
 * (h_B and y in the caller's length unit, s the unit surface
 * FMM_ARRAY_SURFACE):
 *   FMM_WORK_UP    upward equivalent densities rho, a = alpha_inner
 *                  (P2M at leaves, M2M above: "Computational structure
 *                  of FMM operators"), boxes of
 *                  level >= 2; ld = nsurf rounded up to 4;
 *   FMM_WORK_DOWN  downward equivalent densities, a = alpha_outer (after
 *                  M2L, P2L and L2L), boxes of level >= 2; ld as UP;
 *   FMM_WORK_QHAT  compressed multipoles Vk^T rho_up; ld = k rounded up to 16;
 *   FMM_WORK_CHAT  the M2L's output: Uk * chat is the check potential of the
 *                  box's V list on its downward check surface (y' =
 *                  alpha_inner s), boxes with a non-empty V list; ld as QHAT.
 * Rows of boxes a pass does not write hold unspecified values.  Waits for the
 * last evaluation's stream, then copies; FMM_ERR_INVALID_ARG before the
 * first evaluation, for a host-only plan or a short dst.  (Evaluations by
 * fmm_evaluate_noalloc use other memory and are not seen here.) */
enum { FMM_WORK_UP = 0, FMM_WORK_DOWN = 1, FMM_WORK_QHAT = 2, FMM_WORK_CHAT = 3 };
fmm_status fmm_plan_get_workspace(fmm_plan_t plan, int which, void *dst, int64_t bytes,
                                  int64_t *needed);

/* Milliseconds each phase of the last evaluation took, measured with CUDA
 * events on the evaluation stream when timing is on (FMM_TIMING=1 in the
 * environment at plan creation).  phase: 0 upward, 1 M2L, 2 downward,
 * 3 leaf evaluation.  Synchronises the plan's last stream. */
fmm_status fmm_plan_phase_ms(fmm_plan_t plan, int phase, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* KIFMM_H */
