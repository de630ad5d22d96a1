/*
 * plo.h — C ABI of libplo, a GB300 (sm_103a) library that renders complex
 * luminaires stored as plenoctrees and trains / distils the NeRF-SH network
 * they come from.
 *
 * Method: Condor & Jarabo, "A Learned Radiance-Field Representation for
 * Complex Luminaires" (EGSR 2022, arXiv 2207.05009).  A luminaire is a
 * radiance field inside a proxy box (Sec. 3); along a ray r(t) the library
 * returns the emitted radiance L_e (Eq. 3) and the transmittance T(r, t1) so
 * that the caller forms L_o = L_e + T * L_i (Eq. 2, read with the pass-through
 * factor T; alpha = 1 - T is Eq. 5).  The field is stored as a sparse octree
 * of leaves holding a density sigma and real SH coefficients of the emission
 * (Sec. 4.2, Sec. 5).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are caller-owned DEVICE memory (for example PyTorch
 *     tensors on the current device); h_* are caller-owned HOST memory.  The
 *     library never frees caller memory and keeps no pointer to it after the
 *     call returns (asynchronous calls read/write it in stream order).
 *   - Handles (plo_tree) are owned by the library and freed by *_free.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls marked "async" enqueue work and return without
 *     synchronising; errors found on the host are returned immediately.
 *   - On a non-OK status, plo_last_error() returns a message for the calling
 *     thread.  No call aborts the process.
 *   - All arrays are C-contiguous, little-endian, float32 unless stated.
 */
#ifndef PLO_H
#define PLO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLO_OK = 0,
    PLO_ERR_INVALID_ARG = -1,     /* bad pointer, size, enum or parameter value      */
    PLO_ERR_BAD_TREE = -2,        /* canonical tree failed validation                 */
    PLO_ERR_OOM = -3,             /* device or host allocation failed                 */
    PLO_ERR_CUDA = -4,            /* a CUDA runtime call failed                       */
    PLO_ERR_TRAVERSAL_LIMIT = -5, /* some ray hit the per-ray step cap (device-found) */
    PLO_ERR_TIMEOUT = -6,         /* a bounded device wait gave up (device-found)     */
    PLO_ERR_UNSUPPORTED = -7      /* valid request this build does not implement      */
} plo_status;

/* Leaf storage precision (Sec. 5 leaves, stored in FP32 or in 16-bit floats
 * with a per-leaf power-of-two FP32 scale for the SH coefficients). */
enum { PLO_PREC_FP32 = 0, PLO_PREC_FP16 = 1, PLO_PREC_BF16 = 2 };
/* Transmittance model: Beer-Lambert, or the linear model of Eq. 4 with
 * weights w_i = T_i - T_{i+1}, or Eq. 4 integrated literally inside each
 * segment, w_i = (T_i^2 - T_{i+1}^2) / 2. */
enum { PLO_TRANS_EXP = 0, PLO_TRANS_LINEAR = 1, PLO_TRANS_LINEAR_LITERAL = 2 };
/* Emission activation S of Eq. 6: max(0, x), or l_max * sigmoid(x). */
enum { PLO_ACT_RELU = 0, PLO_ACT_SIGMOID = 1 };

/* Proxy geometry (Sec. 5: the luminaire is attached to a sphere or a box).
 * BOX integrates over the part of the ray inside the tree's bounding box;
 * SPHERE over the part inside both that box and the ball `sphere`. */
enum { PLO_PROXY_BOX = 0, PLO_PROXY_SPHERE = 1 };

/* Per-ray status codes written to the optional d_status arrays. */
enum { PLO_RAY_OK = 0, PLO_RAY_STEP_LIMIT = 1, PLO_RAY_INVALID = 3 };

typedef struct plo_tree plo_tree;

/* Canonical host tree (Sec. 5 plenoctree), read-only during the call.
 *   depth      maximum leaf level, 0..16 (level 0 = the root cell).
 *   sh_degree  l_max, 0..4; K = (l_max + 1)^2 coefficients per channel.
 *   child      int32 [n_nodes][8]: >= 0 internal node id, -1 empty octant,
 *              <= -2 leaf with id -c-2.  Node 0 is the root; the child slot is
 *              bx | by << 1 | bz << 2 with b = 1 for the upper half.
 *              n_nodes == 0 means the root itself is leaf 0 (n_leaves == 1) or
 *              the tree is empty (n_leaves == 0).
 *   sigma      float [n_leaves], finite, >= 0 (density per unit length).
 *   sh         float [n_leaves][3][K] channel-major SH coefficients.
 *   bbox_min/max  proxy box in world space the unit cube maps onto. */
typedef struct {
    int32_t depth;
    int32_t sh_degree;
    int64_t n_nodes;
    int64_t n_leaves;
    const int32_t* child;
    const float* sigma;
    const float* sh;
    float bbox_min[3];
    float bbox_max[3];
} plo_tree_desc;

/* Render parameters.  Zero-initialised fields give the exact integral over
 * the proxy box with exponential transmittance and max(0, .) emission.
 *   transmittance  PLO_TRANS_*          activation  PLO_ACT_*
 *   l_max          scale of the sigmoid activation (Eq. 6); ignored for RELU
 *   t_stop         stop a ray once T < t_stop after a leaf (0 = never early;
 *                  alpha_max of Sec. 6.2 is t_stop = 1 - alpha_max)
 *   sigma_min      leaves with sigma < sigma_min count as empty (Sec. 6.2)
 *   max_steps      per-ray cap on cells visited; 0 = 4 * 2^depth + 64
 *   saturate       1: a ray whose final T is below t_stop counts as opaque and
 *                  returns T = 0 (the "saturated" ray of Sec. 6.2); 0: it
 *                  returns the T it reached
 *   proxy          PLO_PROXY_BOX or PLO_PROXY_SPHERE
 *   sphere         sphere proxy centre xyz and radius (world space, radius
 *                  > 0); ignored for PLO_PROXY_BOX.  Not supported by the
 *                  batch entry points (their luminaires use their boxes). */
typedef struct {
    int32_t transmittance;
    int32_t activation;
    float l_max;
    float t_stop;
    float sigma_min;
    int32_t max_steps;
    int32_t saturate;
    int32_t proxy;
    float sphere[4];
} plo_render_params;

/* Device layout of a packed tree (plo_build_tree_ex).
 *   PLO_LAYOUT_OCTREE  the octree itself: 8-byte child entries, a leaf's
 *                      density in its parent's entry; the render walks it
 *                      cell by cell with a descent per cell.
 *   PLO_LAYOUT_BRICKS  the octree above level depth - s, and below it dense
 *                      bricks of (2^s)^3 finest cells holding the entry of
 *                      the leaf that covers each cell; the render walks the
 *                      bricks with a per-axis digital differential analyser
 *                      (one integer step per finest cell, no descent).
 * Both give the same integral (a leaf crossed in several finest cells is
 * the sum of its parts); lookup and trace always use the octree. */
enum { PLO_LAYOUT_OCTREE = 0, PLO_LAYOUT_BRICKS = 1, PLO_LAYOUT_DEFAULT = PLO_LAYOUT_OCTREE };

/* Options of plo_build_tree_ex: precision PLO_PREC_*, layout PLO_LAYOUT_*,
 * brick_log the brick side's log2 (1..3; 0 = 3, 8^3 cells), capped at
 * depth - 1 so that the root is always a node. */
typedef struct {
    int32_t precision;
    int32_t layout;
    int32_t brick_log;
} plo_build_options;

typedef struct {
    int32_t depth, sh_degree, precision;
    int32_t top_levels;        /* levels staged in shared memory by the render kernel */
    int64_t n_nodes, n_leaves;
    int64_t n_sh_records;      /* leaves with at least one non-zero SH coefficient   */
    int64_t node_bytes;        /* device bytes of the node table                     */
    int64_t sh_bytes;          /* device bytes of the SH record table                */
    int32_t sh_record_stride;  /* bytes between SH records                           */
    int32_t device;            /* CUDA device that holds the tree                    */
    int32_t layout;            /* PLO_LAYOUT_*                                       */
    int32_t brick_log;         /* brick side log2 (0 for the octree layout)         */
    int64_t n_bricks;          /* bricks of the brick layout                         */
    int64_t brick_bytes;       /* device bytes of the bricks                         */
    int64_t top_nodes;         /* nodes of the brick layout's top tree               */
} plo_tree_info;

/* Checks a canonical tree on the host without touching a GPU: index ranges,
 * each node and leaf referenced at most once (no cycles or sharing), node
 * levels below `depth`, finite non-negative sigma, finite SH, box extents.
 * Returns PLO_OK, PLO_ERR_INVALID_ARG, PLO_ERR_BAD_TREE, or PLO_ERR_OOM when
 * the host cannot hold the per-node and per-leaf flags for the given counts. */
plo_status plo_validate_tree(const plo_tree_desc* desc);

/* Validates `desc`, packs it into the device layout at `precision`
 * (PLO_PREC_*) and uploads it to the current CUDA device.  Synchronous.
 * FP16 / BF16 store each leaf's SH coefficients as binary16 / bfloat16 times a
 * per-leaf power-of-two FP32 scale, and sigma as a 24-bit float (8-bit
 * exponent, 16-bit mantissa, round-to-nearest-even).  On success *out owns the device copy; free it with
 * plo_tree_free.  The host arrays may be released after the call.  Packing
 * runs on all host cores.  Errors: those of plo_validate_tree;
 * PLO_ERR_INVALID_ARG for a bad precision; PLO_ERR_OOM when a host or device
 * allocation fails (nothing of the tree is left allocated); PLO_ERR_CUDA. */
plo_status plo_build_tree(const plo_tree_desc* desc, int32_t precision, plo_tree** out);

/* plo_build_tree with a chosen layout (plo_build_tree uses PLO_LAYOUT_DEFAULT,
 * the octree: on the depth-10 luminaire it renders ~1.5x faster than bricks,
 * whose walk splits a warp between brick and octree steps).  Same errors, plus PLO_ERR_INVALID_ARG for an unknown
 * layout or brick_log.  The brick layout keeps the octree node table too
 * (for lookup and trace), so it takes node_bytes + brick_bytes. */
plo_status plo_build_tree_ex(const plo_tree_desc* desc, const plo_build_options* options, plo_tree** out);

/* Frees a tree (NULL is a no-op).  Synchronises the device first. */
void plo_tree_free(plo_tree* tree);

plo_status plo_tree_get_info(const plo_tree* tree, plo_tree_info* out);

/* Renders n rays (async).  Per ray, paper Eq. 3-5: clip to the proxy,
 * walk the octree front to back over exact per-leaf segments, evaluate the
 * leaf's SH emission in the ray direction, composite emission/absorption.
 *   d_rays    float [n][6]: origin xyz, direction xyz (world space; the
 *             direction should be unit length: t is measured in its units).
 *   d_rgb     float [n][3] emitted radiance L_e.
 *   d_T       float [n] transmittance T(r, t1); alpha = 1 - T.
 *   d_status  int32 [n] per-ray PLO_RAY_* code, or NULL.
 * A ray with a NaN/Inf component or a zero direction gets NaN outputs and
 * PLO_RAY_INVALID.  A ray that exceeds max_steps keeps its partial result,
 * gets PLO_RAY_STEP_LIMIT and raises the tree's device error flag (read by
 * plo_tree_check).  n == 0 is a no-op.  Calls with n >= 2^20 take an 8-byte
 * work counter from the stream-ordered allocator (cudaMallocAsync on
 * `stream`), so that warps claim rays dynamically. */
plo_status plo_render_rays(const plo_tree* tree, const float* d_rays, int64_t n, const plo_render_params* params,
                           float* d_rgb, float* d_T, int32_t* d_status, void* stream);

/* Same computation as plo_render_rays for rays in HOST memory: copies
 * h_rays to the device, renders, copies h_rgb / h_T back, in chunks that
 * overlap copies with rendering on internal streams ordered after `stream`.
 * Synchronous (returns after h_rgb / h_T are written).  Pinned host memory
 * gives full copy bandwidth; pageable memory works but is slower. */
plo_status plo_render_rays_host(const plo_tree* tree, const float* h_rays, int64_t n,
                                const plo_render_params* params, float* h_rgb, float* h_T, void* stream);

/* Allocation-free variant of plo_render_rays_host, for callers that cannot
 * allocate device memory while they render: for example a CPU path tracer
 * that queries the luminaire from its emitter code inside the frame loop, or
 * a host process whose device memory is fixed at start-up.  Same inputs,
 * outputs and results as plo_render_rays_host; the paper has no counterpart.
 *   - Rays and results are staged in a fixed device array inside the library
 *     (10 MiB, held by every GPU that loads the library until exit), so at
 *     most 262,144 rays per call; larger n returns PLO_ERR_INVALID_ARG.
 *   - After the set-up call below, a call makes no device allocation and no
 *     allocating library call.
 *   - The first call in a CUDA context (once per device, and again after
 *     that device's context is reset) looks up the array's device address.
 *     With lazy module loading (CUDA_MODULE_LOADING=LAZY, the runtime's
 *     default) that lookup may also load the library's device code and with
 *     it the 10 MiB array: the first call per context is the set-up step, so
 *     make it at start-up and before capturing any stream.  Later calls make
 *     no device allocation.
 *   - All calls share the array: calls whose work overlaps on the GPU (other
 *     streams, other host threads) race and corrupt each other's results.
 *   - Copies and the render run on `stream`; the call returns after h_rgb and
 *     h_T are written.  The tree must live on the current device. */
plo_status plo_render_rays_host_noalloc(const plo_tree* tree, const float* h_rays, int64_t n,
                                        const plo_render_params* params, float* h_rgb, float* h_T, void* stream);

/* ------------------------------------------------------------------------
 * Batched render of several luminaires (one launch for all of them).
 * Rays of tree t are d_rays[ray_offsets[t] .. ray_offsets[t+1]) of one
 * concatenated array (outputs likewise).  A persistent kernel drains one
 * queue of ray claims over all trees, so uneven ray counts balance
 * themselves; trees may differ in depth, SH degree and leaf precision.
 * The batch keeps pointers to the trees: they must outlive it. */
typedef struct plo_batch plo_batch;

/* Launch shape of the batch kernel.
 *   claim_rays     rays a warp takes from the queue at a time (multiple of 32)
 *   blocks_per_sm  resident blocks per SM (0: as many as fit)
 *   top_nodes      nodes per tree staged in shared memory (0..73) */
typedef struct {
    int32_t claim_rays;
    int32_t blocks_per_sm;
    int32_t top_nodes;
} plo_batch_config;

/* n_trees in [1, 16]; ray_offsets: host int64 [n_trees + 1], starting at 0. */
plo_status plo_batch_create(const plo_tree* const* trees, int32_t n_trees, const int64_t* ray_offsets,
                            const plo_render_params* params, plo_batch** out);
void plo_batch_free(plo_batch* batch);
plo_status plo_batch_set_config(plo_batch* batch, const plo_batch_config* cfg);
plo_status plo_batch_get_config(const plo_batch* batch, plo_batch_config* cfg);

/* Renders the whole batch (async): d_rays float [n][6], d_rgb float [n][3],
 * d_T float [n], d_status int32 [n] or NULL, n = ray_offsets[n_trees]. */
plo_status plo_batch_render(plo_batch* batch, const float* d_rays, float* d_rgb, float* d_T, int32_t* d_status,
                            void* stream);

/* Captures one batch render on these buffers into a CUDA graph (queue reset
 * + kernel); plo_batch_replay launches it on `stream` (async).  Changing the
 * config drops the graph. */
plo_status plo_batch_capture(plo_batch* batch, const float* d_rays, float* d_rgb, float* d_T, int32_t* d_status,
                             void* stream);
plo_status plo_batch_replay(plo_batch* batch, void* stream);

/* Times every launch shape of a small grid (claim 32..1024, blocks per SM,
 * shared-memory staging on/off) on these buffers, `reps` launches each, and
 * keeps the fastest; returns it and its time per launch.  Synchronous. */
plo_status plo_batch_autotune(plo_batch* batch, const float* d_rays, float* d_rgb, float* d_T, int32_t reps,
                              void* stream, plo_batch_config* best, float* best_ms);

/* Point -> leaf lookup (async), the descent step of the render.
 *   d_points  float [n][3] in the tree's unit-cube coordinates.
 *   d_dirs    float [n][3] or NULL: on a cell plane a point belongs to the
 *             upper cell when the direction component is >= 0 (always, when
 *             NULL); the faces of the root cube are closed.
 *   d_leaf    int64 [n] canonical leaf id, -1 for an empty octant, -2 outside
 *             the unit cube.
 *   d_level   int32 [n] level of the cell found, or NULL. */
plo_status plo_lookup_points(const plo_tree* tree, const float* d_points, const float* d_dirs, int64_t n,
                             int64_t* d_leaf, int32_t* d_level, void* stream);

/* Diagnostic trace (async): the first `max_cells` cells each ray crosses, in
 * order, exactly as plo_render_rays walks them.
 *   d_leaf   int64 [n][max_cells] canonical leaf id, -1 for an empty octant
 *            (unused slots -3).
 *   d_t      float [n][max_cells][2] segment [t_in, t_out] along the ray.
 *   d_count  int32 [n] number of cells crossed (may exceed max_cells). */
plo_status plo_trace_rays(const plo_tree* tree, const float* d_rays, int64_t n, const plo_render_params* params,
                          int32_t max_cells, int64_t* d_leaf, float* d_t, int32_t* d_count, void* stream);

/* Synchronises `stream` and reports device-detected errors of earlier
 * renders of this tree: PLO_ERR_TRAVERSAL_LIMIT if some ray hit its step cap.
 * Clears the flag. */
plo_status plo_tree_check(const plo_tree* tree, void* stream);

/* ------------------------------------------------------------------------
 * Learned part (Sec. 4.2-4.4): the NeRF-SH network and its training.
 *
 * Network: positional encoding of the sample position x in the unit cube,
 * gamma(x) = [x, sin(2^j pi x), cos(2^j pi x)]_{j<10} (63 features), eight
 * fully connected layers of 256 with ReLU (the trunk), then the output
 * layers of the chosen architecture:
 *   PLO_ARCH_LINEAR_HEAD  one linear layer 256 -> 1 + 3K (sigma_raw, SH);
 *   PLO_ARCH_PAPER        a 128-wide hidden layer before the SH outputs
 *                         (Sec. 4.2): sigma_raw = w_s . h8 + b_s and
 *                         SH = W_c ReLU(W_f h8 + b_f) + b_c (128 -> 3K).
 * sigma = ReLU(sigma_raw); emission = l_max * sigmoid(sum_k c_k Y_k(d))
 * (Eq. 6); SH coefficients channel-major.  BF16 weights and activations,
 * FP32 accumulation on the tensor cores, FP32 master weights.  Parameters
 * are exchanged in a canonical FP32 order of (W [out][in], b [out]) blocks:
 * the trunk's 8 layers (in 63, then 256), then LINEAR_HEAD: the head
 * (1 + 3K x 256); PAPER: sigma (1 x 256), the 128-wide layer (128 x 256),
 * the SH layer (3K x 128).  Rays for training are given in the unit cube
 * (the proxy box). */
typedef struct plo_mlp plo_mlp;

/* Output architecture (plo_mlp_desc.arch). */
enum { PLO_ARCH_LINEAR_HEAD = 0, PLO_ARCH_PAPER = 1 };

/* Loss of Sec. 4.3 on values divided by l_max: PAPER = sum over channels of
 * ((C^ - C) / (C^ + eps))^2 (denominator held constant) + (alpha^ - alpha)^2
 * (Eq. 7-9); REG = the colour term only; MSE = plain squared error. */
enum { PLO_LOSS_PAPER = 0, PLO_LOSS_REG = 1, PLO_LOSS_MSE = 2 };

typedef struct {
    int32_t sh_degree;      /* must be 3 (48 SH coefficients)                      */
    int32_t transmittance;  /* PLO_TRANS_EXP or PLO_TRANS_LINEAR                   */
    int32_t loss;           /* PLO_LOSS_*                                          */
    int32_t total_steps;    /* learning-rate decay horizon                         */
    float l_max;            /* maximum radiance: sigmoid scale and loss unit       */
    float eps;              /* loss regulariser, 0.01 in the paper                 */
    float lr0, lr1;         /* exponential decay lr0 -> lr1 (5e-4 -> 5e-6)         */
    float init_radiance;    /* emission the network starts from (0: l_max / 2)     */
    int32_t arch;           /* PLO_ARCH_LINEAR_HEAD or PLO_ARCH_PAPER               */
    uint64_t seed;          /* stream of the stratified-sampling and distillation
                               jitter                                              */
} plo_mlp_desc;

/* Number of parameters of the network for SH degree `sh_degree`:
 * plo_mlp_param_count for PLO_ARCH_LINEAR_HEAD; _arch for either (-1 for an
 * unknown arch). */
int64_t plo_mlp_param_count(int32_t sh_degree);
int64_t plo_mlp_param_count_arch(int32_t sh_degree, int32_t arch);

/* Creates the network on the current device.  Initial parameters (drawn
 * from `seed`): He-uniform hidden weights and zero hidden biases; the
 * weights that produce sigma and SH He-uniform scaled by 0.1, sigma bias 0.5
 * (every sample starts with positive density), and the DC SH bias of each
 * channel set so that the emission starts at init_radiance.  Starting at l_max / 2 against HDR
 * targets far below l_max, the first updates drive sigma below zero
 * everywhere and the ReLU keeps it there. */
plo_status plo_mlp_create(const plo_mlp_desc* desc, uint64_t seed, plo_mlp** out);
void plo_mlp_free(plo_mlp* mlp);

/* Host <-> device parameter exchange in the canonical order (n must equal
 * plo_mlp_param_count).  Synchronous.  get_grads returns the gradient of the
 * last training step (the one its Adam update used). */
plo_status plo_mlp_set_params(plo_mlp* mlp, const float* h_params, int64_t n);
plo_status plo_mlp_get_params(const plo_mlp* mlp, float* h_params, int64_t n);
plo_status plo_mlp_get_grads(const plo_mlp* mlp, float* h_grads, int64_t n);

/* Raw network outputs at n points (async).  d_points float [n][3] in the
 * unit cube; d_raw float [n][1 + 3K] (sigma_raw, then SH coefficients). */
plo_status plo_mlp_forward(plo_mlp* mlp, const float* d_points, int64_t n, float* d_raw, void* stream);

/* One training step (async): stratified samples along each ray (Sec. 4.1),
 * network forward, quadrature render (Eq. 3-5), the loss, backward, Adam
 * with the decayed learning rate (Sec. 4.4).
 *   d_rays      float [n_rays][6] origin, direction (unit-cube coordinates)
 *   d_rgb_gt    float [n_rays][3] target L_e;  d_alpha_gt float [n_rays]
 *   n_samples   32, 64, 128 or 256; n_rays * n_samples a multiple of 128
 *   d_jitter    float [n_rays][n_samples] in [0,1), or NULL to draw it from
 *               the desc's seed and the step number (SplitMix64)
 *   d_loss_out  float [1]: the batch's mean loss before the update. */
plo_status plo_mlp_train_step(plo_mlp* mlp, const float* d_rays, const float* d_rgb_gt, const float* d_alpha_gt,
                              int32_t n_rays, int32_t n_samples, const float* d_jitter, float* d_loss_out,
                              void* stream);

/* One step of the paper's coarse/fine training (Sec. 4.3-4.4, Eq. 7) on two
 * networks with the same l_max, transmittance and loss (async):
 *   coarse: n_coarse stratified samples (jitter as in plo_mlp_train_step),
 *           loss L_c = the colour term (PAPER trains the coarse network with
 *           REG; MSE and REG train both networks with that loss);
 *   fine:   the coarse samples plus n_fine samples drawn from the coarse
 *           weights: coarse sample i owns [t_i, t_{i+1}) (the last one ends
 *           at the exit), the density is constant there with mass
 *           proportional to w_i + 1e-5, and u_j = (j + xi_j) / n_fine goes
 *           through the inverse CDF; the network is trained on all
 *           n_coarse + n_fine samples in ascending order with L_f + L_alpha.
 * No gradient flows through the placement.  Each network takes one Adam
 * step.  n_coarse, n_fine multiples of 32, n_coarse <= 128, n_coarse +
 * n_fine in {64, 96, 128, 192, 256} (the paper: 64 + 128); n_rays *
 * n_coarse a multiple of 128.  d_xi float [n_rays][n_fine] in [0,1), or NULL
 * to draw it from the fine network's seed.  d_loss_out float [1]: mean over
 * rays of L_c + L_f + L_alpha before the updates. */
plo_status plo_mlp_train_step_hier(plo_mlp* coarse, plo_mlp* fine, const float* d_rays, const float* d_rgb_gt,
                                   const float* d_alpha_gt, int32_t n_rays, int32_t n_coarse, int32_t n_fine,
                                   const float* d_jitter, const float* d_xi, float* d_loss_out, void* stream);

/* The fine-sample placement of plo_mlp_train_step_hier alone (async), for
 * testing: given the coarse parameters d_t, lengths d_delta and weights d_w
 * (float [n_rays][n_coarse]) and d_xi (float [n_rays][n_fine]), writes the
 * merged parameters d_t_out and lengths d_delta_out (float [n_rays][n_coarse
 * + n_fine], ascending; the last length ends where the ray leaves the unit
 * cube, 0 for rays that miss it). */
plo_status plo_hier_samples(const float* d_rays, int32_t n_rays, int32_t n_coarse, int32_t n_fine, const float* d_t,
                            const float* d_delta, const float* d_w, const float* d_xi, float* d_t_out,
                            float* d_delta_out, void* stream);

/* Distils the network into a plenoctree (Sec. 5, "Creating the plenoctree";
 * synchronous).  Every voxel of the 2^depth grid (depth 1..10) is evaluated
 * at its centre; voxels with sigma >= sigma_thresh (0.01 in the paper) are
 * kept, each as a leaf holding the mean of ReLU(sigma_raw) and of the raw SH
 * coefficients over `samples` (1..256) jittered positions inside it (offsets
 * from SplitMix64 keyed by the desc's seed and the voxel's Morton code).  The
 * tree is packed at `precision` in the octree layout, on the device (no host
 * copy of the leaves), and owned by *out; render it with PLO_ACT_SIGMOID and
 * the network's l_max.  Device memory: 4 bytes per voxel of the 2^depth grid
 * for the kept codes, per kept voxel 5 bytes plus its SH record (12K bytes
 * FP32, 6K 16-bit, rounded up to 16), the node tables (96 bytes per node),
 * plus the network's workspace.
 * Errors: PLO_ERR_INVALID_ARG; PLO_ERR_OOM when a host or device allocation
 * fails; PLO_ERR_CUDA; PLO_ERR_TIMEOUT from the network's kernels. */
plo_status plo_distill(plo_mlp* mlp, int32_t depth, int32_t samples, float sigma_thresh, int32_t precision,
                       plo_tree** out, void* stream);

/* Checkpoint of a network and its training state (Sec. 4.4 training runs for
 * days; an interrupted run resumes where it stopped).  plo_mlp_save writes,
 * synchronously, to a file at `path`:
 *   "PLOMLP01", a uint64 header length H, an H-byte flat JSON header (format
 *   "plo-mlp", version 1, the plo_mlp_desc fields, seed as a decimal string,
 *   the step count, n_params, and the byte offset of each blob), then the
 *   blobs at 64-byte-aligned offsets, little-endian: "master", "adam_m",
 *   "adam_v" (float32 [n_params] each in the canonical parameter order of
 *   plo_mlp_get_params: FP32 weights and Adam's first and second moments)
 *   and "weights_bf16" (bfloat16 copies of every weight matrix, canonical
 *   order, no biases).
 * The sample jitter is keyed by (seed, step), so seed and step restore the
 * training's random stream.  plo_mlp_load creates a network on the current
 * device from such a file (the caller frees it with plo_mlp_free); it checks
 * the header, the sizes and that the bf16 copies are the rounding of the FP32
 * weights.  plo_mlp_checkpoint_info reads and checks only the header, on the
 * host (no GPU), returning its description and step (either may be NULL).
 * Errors: PLO_ERR_INVALID_ARG for an unreadable, truncated or inconsistent
 * file; PLO_ERR_UNSUPPORTED for another format version; PLO_ERR_OOM. */
plo_status plo_mlp_save(const plo_mlp* mlp, const char* path);
plo_status plo_mlp_load(const char* path, plo_mlp** out);
plo_status plo_mlp_checkpoint_info(const char* path, plo_mlp_desc* desc, int64_t* step);

/* Test hooks of the training step (async), so that each stage can be compared
 * with a reference element by element.
 * plo_mlp_get_activation: copies rows [0, n_rows) of the bf16 input of
 *   network layer `layer` as the last forward or training step left it:
 *   layer 0 is the positional encoding (64 columns, column 63 zero),
 *   1..8 the outputs of the eight trunk layers (256 columns), and for
 *   PLO_ARCH_PAPER 9 the 128-wide layer's output; PLO_MLP_DZ_BASE + l (l =
 *   0..7) the last training step's d loss / d Z_l, the gradient at the
 *   pre-activation of trunk layer l (256 columns).  d_out bf16 [n_rows][cols].
 * plo_mlp_quad: the quadrature render and loss stage of plo_mlp_train_step
 *   alone (Eq. 3-9, the network's l_max, eps, transmittance and loss) on
 *   given raw outputs d_raw float [n_rays * n_samples][1 + 3K] (row
 *   ray * n_samples + j) and segment lengths d_delta float [n_rays *
 *   n_samples].  Writes d_ray_out float [n_rays][5] (C^ rgb, alpha^, the
 *   ray's loss) and, if d_draw is not NULL, d (mean loss) / d raw float
 *   [n_rays * n_samples][1 + 3K] as the backward pass receives it (rounded
 *   to bf16).  n_samples in {32, 64, 96, 128, 192, 256}. */
enum { PLO_MLP_DZ_BASE = 16 };
plo_status plo_mlp_get_activation(const plo_mlp* mlp, int32_t layer, void* d_out, int64_t n_rows, void* stream);
plo_status plo_mlp_quad(plo_mlp* mlp, const float* d_rays, const float* d_raw, const float* d_delta,
                        const float* d_rgb_gt, const float* d_alpha_gt, int32_t n_rays, int32_t n_samples,
                        float* d_ray_out, float* d_draw, void* stream);

/* Canonical export of a packed tree (synchronous): the node table as the
 * canonical child table (node ids of the packed layout; leaves by their
 * canonical ids), and every leaf's sigma and SH coefficients, dequantised for
 * FP16 / BF16 trees.  h_child int32 [n_nodes][8], h_sigma float [n_leaves],
 * h_sh float [n_leaves][3][K] (counts from plo_tree_get_info).  A distilled
 * tree exported this way and rebuilt with plo_build_tree renders the same. */
plo_status plo_tree_export(const plo_tree* tree, int32_t* h_child, float* h_sigma, float* h_sh);

/* Synchronises `stream`; PLO_ERR_TIMEOUT if a tensor-core kernel gave up on
 * a bounded pipeline wait since the last check (the flag is cleared). */
plo_status plo_mlp_check(const plo_mlp* mlp, void* stream);

/* Number of training steps taken. */
int64_t plo_mlp_step(const plo_mlp* mlp);

/* The tensor-core building blocks (async), exposed for testing.
 * plo_gemm_bf16: C[M][N] = A[M][K] B[N][K]^T, A and B bf16 row-major, bias
 *   16-byte aligned,
 *   (N, K) in {(256, 64), (256, 256), (64, 256)}; epilogue 0: bf16
 *   ReLU(C + bias), and if d_bits is not NULL where C + bias > 0 (fp32,
 *   before rounding) as bits (uint32 [M][N / 32], bit j of word c for
 *   column 32 c + j); 1: fp32
 *   C + bias; 2: bf16 C * (mask > 0) with mask bf16 [M][N]; 3: bf16 C with
 *   the columns whose bit in d_bits is clear set to 0; d_out row-major
 *   [M][N].
 * plo_wgrad_bf16: dW[n_out][n_in] += dZ^T H over M rows (dZ bf16 [M][n_out],
 *   H bf16 [M][n_in], n_out, n_in in {64, 256}, M a multiple of 64); if
 *   d_db (fp32 [n_out]) is not NULL, also d_db[o] += sum_m dZ[m][o], the
 *   bias gradient, from the same pass over dZ.
 * d_err: device word, bit 1 set if a pipeline wait gave up. */
plo_status plo_gemm_bf16(const void* d_A, const void* d_B, int32_t M, int32_t N, int32_t K, int32_t epilogue,
                         const float* d_bias, const void* d_mask, uint32_t* d_bits, void* d_out, unsigned int* d_err,
                         void* stream);
plo_status plo_wgrad_bf16(const void* d_dZ, int32_t n_out, const void* d_H, int32_t n_in, int32_t M, float* d_dW,
                          float* d_db, unsigned int* d_err, void* stream);

/* ------------------------------------------------------------------------
 * The luminaire as an emitter in a path tracer (Sec. 3 Eq. 2: what leaves
 * the proxy is L_o = L_e + T L_i; Sec. 5 "Sampling": the proxy surface is
 * sampled uniformly).
 *
 * Scene: a closed room (axis-aligned box, diffuse walls seen from inside)
 * holding the luminaire; the proxy is the tree's bounding box, which must
 * lie inside the room.  Per path (pixel p % (width * height) of sample
 * p / (width * height)), with uniforms u[0 .. 2 + 5 * max_bounces):
 *   camera ray through pixel (px + u0, py + u1) of a pinhole camera
 *   (cam_pos looking at cam_target, cam_up, vertical field of view fov_y);
 *   per bounce b (u[2+5b] picks a proxy face by area, u[3+5b], u[4+5b] a
 *   point y on it, u[5+5b], u[6+5b] the bounce):
 *     the luminaire along the ray: camera rays add its L_e; the throughput
 *       is multiplied by its T (light from behind passes through);
 *     wall point x, inward normal n, albedo rho of that wall (walls
 *       x-, x+, y-, y+, z-, z+);
 *     next event: if y's face faces x, add
 *       thr * rho / pi * L_e(x -> y) * cos_x * cos_y / |y - x|^2 * A
 *       (A: proxy surface area; L_e(x -> y) the luminaire's emission along
 *       the ray from x through y);
 *     cosine-weighted bounce about n (u5 -> cos^2 of the polar angle
 *       1 - u5, u6 -> azimuth), thr *= rho.
 * emitter PLO_PT_OCTREE queries the tree (plo_render_rays with `params`);
 * PLO_PT_CONSTANT_BOX replaces it by an opaque box of radiance
 * box_radiance, the "explicitly handled" emitter the overhead is measured
 * against. */
enum { PLO_PT_OCTREE = 0, PLO_PT_CONSTANT_BOX = 1 };

typedef struct {
    float room_min[3], room_max[3];
    float albedo[6][3];
    float cam_pos[3], cam_target[3], cam_up[3];
    float fov_y;               /* radians, in (0, 3.1)                  */
    int32_t width, height;
    int32_t max_bounces;       /* 1 .. 16                               */
    int32_t emitter;           /* PLO_PT_*                              */
    float box_radiance[3];     /* PLO_PT_CONSTANT_BOX only              */
} plo_pt_scene;

/* Renders spp samples per pixel (async on `stream`).
 *   params      luminaire queries (PLO_PROXY_BOX only)
 *   d_uniforms  float [spp * width * height][2 + 5 * max_bounces] in [0, 1),
 *               or NULL to draw them from `seed` (SplitMix64)
 *   d_image     float [height][width][3]: mean radiance over the samples
 *   d_samples   float [spp][height][width][3] per-sample radiance, or NULL
 * Allocates its wavefront buffers with cudaMallocAsync on `stream`. */
plo_status plo_pt_render(const plo_tree* lum, const plo_render_params* params, const plo_pt_scene* scene,
                         int32_t spp, uint64_t seed, const float* d_uniforms, float* d_image, float* d_samples,
                         void* stream);

/* ------------------------------------------------------------------------
 * Direct optimisation of the octree's leaves (Sec. 7, "Limitations --
 * Precomputation cost": fitting the SH octree itself, with a total-variation
 * regulariser against aliasing, instead of training a network and projecting
 * it).  The tree's structure is fixed; per leaf i the parameters are a raw
 * density s_i (sigma_i = max(0, s_i)) and the 3K SH coefficients
 * (channel-major), emitting L_max sigmoid(sum_k k_k Y_k(d)) as the network
 * does (Eq. 6).  Each ray is rendered over the exact leaf segments of the
 * octree walk (plo_trace_rays of the structure, Eq. 3-5), so the forward pass
 * equals plo_render_rays of the exported tree with PLO_ACT_SIGMOID.
 * Objective: the paper's loss (Sec. 4.3, as plo_mlp_desc.loss, on values
 * divided by l_max) averaged over the batch's rays, plus
 * tv_sigma TV(s) + tv_sh TV(k), where per leaf and channel the TV term is
 * sqrt(1e-8 + sum_a (x_{n_a(i)} - x_i)^2) over the axes a, n_a(i) being the
 * leaf that holds the point just across i's upper face a at the face's
 * centre (none: outside the cube or an empty octant, the difference is 0),
 * averaged over the leaves.  Adam (beta 0.9, 0.999, eps 1e-8) with step
 * sizes lr * lr_decay^(min(t - 1, total_steps) / total_steps) at update t. */
typedef struct plo_octopt plo_octopt;

typedef struct {
    int32_t transmittance;  /* PLO_TRANS_EXP or PLO_TRANS_LINEAR               */
    int32_t loss;           /* PLO_LOSS_*                                      */
    float l_max;            /* emission scale L_max and loss unit (> 0)        */
    float eps;              /* loss regulariser (0.01 in the paper)            */
    float lr_sigma, lr_sh;  /* Adam step sizes of the densities and the SH     */
    float lr_decay;         /* factor the step sizes fall by over total_steps,
                               in (0, 1]                                       */
    int32_t total_steps;    /* decay horizon (>= 1)                            */
    float tv_sigma, tv_sh;  /* weights of the TV terms (>= 0)                  */
    int64_t max_rays;       /* rays per step the scratch is sized for (>= 1)   */
    int32_t max_cells;      /* cells per ray the trace holds; 0 = 3 * 2^depth
                               + 2 (no ray crosses more)                       */
} plo_octopt_config;

/* What plo_octopt_read / _write move. */
enum {
    PLO_OCTOPT_SIGMA = 0,      /* float [n_leaves]: raw densities s          */
    PLO_OCTOPT_SH = 1,         /* float [n_leaves][3][K]                      */
    PLO_OCTOPT_GRAD_SIGMA = 2, /* float [n_leaves]: d objective / d s of the
                                  last plo_octopt_grad or _step (read only)   */
    PLO_OCTOPT_GRAD_SH = 3,    /* float [n_leaves][3][K] (read only)          */
    PLO_OCTOPT_NEIGHBOURS = 4  /* int32 [n_leaves][3]: n_a(i), -1 for none
                                  (read only)                                 */
};

/* Creates an optimiser on the current device for the structure of `init`
 * (validated as for plo_build_tree; depth <= 10, n_leaves < 2^31), starting
 * from its sigma (as raw densities) and SH coefficients.  Builds the
 * structure's walk tree, the face-neighbour table and its reverse, and
 * allocates the parameters, gradients, Adam moments, the TV scratch (8
 * bytes per coefficient) and the trace scratch (max_rays * cells * 16
 * bytes).  Synchronous.  Errors: those of plo_build_tree;
 * PLO_ERR_INVALID_ARG for a bad config; PLO_ERR_UNSUPPORTED for depth > 10
 * or 2^31 leaves or more; PLO_ERR_OOM. */
plo_status plo_octopt_create(const plo_tree_desc* init, const plo_octopt_config* config, plo_octopt** out);
void plo_octopt_free(plo_octopt* opt);

/* The objective's gradient on n rays (async on `stream`), into the
 * optimiser's gradient buffers (no update).
 *   d_rays      float [n][6] world-space origin and direction
 *   d_rgb_gt    float [n][3] target L_e;  d_alpha_gt float [n] target alpha
 *   d_ray_out   float [n][5] (C^ rgb, alpha^, the ray's loss), or NULL
 *   d_loss_out  float [3] (mean loss, TV(s), TV(k)), or NULL
 * n <= max_rays.  A ray that crosses more than max_cells cells is left out
 * and flagged (plo_octopt_check). */
plo_status plo_octopt_grad(plo_octopt* opt, const float* d_rays, const float* d_rgb_gt, const float* d_alpha_gt,
                           int64_t n, float* d_ray_out, float* d_loss_out, void* stream);

/* plo_octopt_grad followed by one Adam update of every parameter (async).
 * n == 0 is a no-op. */
plo_status plo_octopt_step(plo_octopt* opt, const float* d_rays, const float* d_rgb_gt, const float* d_alpha_gt,
                           int64_t n, float* d_ray_out, float* d_loss_out, void* stream);

/* Copies one of the PLO_OCTOPT_* arrays to `dst` / from `src` (host or
 * device memory; async on `stream`, so a host buffer must outlive the
 * copy).  Writing resets nothing else (Adam's moments stay). */
plo_status plo_octopt_read(const plo_octopt* opt, int32_t what, void* dst, void* stream);
plo_status plo_octopt_write(plo_octopt* opt, int32_t what, const void* src, void* stream);

/* Synchronises `stream`; PLO_ERR_TRAVERSAL_LIMIT if a ray of an earlier
 * step crossed more than max_cells cells (the flag is cleared). */
plo_status plo_octopt_check(plo_octopt* opt, void* stream);

/* Packs the current parameters into a renderable tree (synchronous):
 * sigma = max(0, s) and the coefficients, on the structure of `init`.
 * Render it with PLO_ACT_SIGMOID and the optimiser's l_max. */
plo_status plo_octopt_build_tree(const plo_octopt* opt, const plo_build_options* options, plo_tree** out);

/* ------------------------------------------------------------------------
 * Test hooks for failure detection (nothing here faults or hangs a GPU).
 * plo_debug_fail_alloc_after(n): the n-th following device allocation made
 *   by the library fails as out-of-memory (n < 0 turns the hook off).
 * plo_debug_gemm_stall: launches the tensor-core GEMM (N = 256, K = 64) with
 *   a producer that issues no loads, so every pipeline wait gives up after
 *   `wait_limit` polls; the kernel sets bit 1 of *d_err, frees its TMEM and
 *   returns, leaving the context usable.  Async. */
void plo_debug_fail_alloc_after(int32_t n);
plo_status plo_debug_gemm_stall(const void* d_A, const void* d_B, int32_t M, void* d_out, unsigned int* d_err,
                                uint32_t wait_limit, void* stream);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* plo_last_error(void);

/* Library version string. */
const char* plo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PLO_H */
