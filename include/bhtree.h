/*
 * bhtree.h -- C ABI of the GB300 tree-code force evaluation
 * (N. Nakasato, "Implementation of a Parallel Tree Method on a GPU").
 *
 * The library evaluates softened gravitational accelerations and potentials
 * (Eq. 1) with the tree method of Sec. 4: a Morton ordering of the particles
 * (Sec. 5), an octree with monopole (and optionally quadrupole) cell moments
 * (Sec. 4.1, 4.4), a tree walk with the modified opening criterion of Eq. (2),
 * and softened particle-cell / particle-particle interactions.  Every step
 * runs in hand-written sm_103a kernels; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - pointers named d_* are DEVICE pointers on the context's device; h_* are
 *     host pointers; nothing else is accepted.
 *   - particles are float4 records (x, y, z, m), 16-byte aligned, n of them;
 *     results are float4 records (ax, ay, az, phi) in the caller's order, with
 *     attractive accelerations and phi = -sum m_j / sqrt(r^2 + eps^2) (the
 *     paper's p_i is -phi_i).  Gravitational constant G = 1.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous: they only enqueue
 *     work.  Device-side failures (non-finite input, capacity, a wait that
 *     timed out) are recorded in the context's status word and returned by the
 *     next bh_status() / bh_stats() call, which synchronise the stream.
 *   - the caller owns every pointer it passes; the context owns its workspace.
 *   - return value: BH_OK (0) or a negative BH_ERR_* code; bh_strerror()
 *     names it.  Argument errors are reported before anything is enqueued.
 */
#ifndef BHTREE_H
#define BHTREE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BH_OK = 0,
    BH_ERR_INVALID = -1,        /* bad argument (null, misaligned, n < 0, bad theta/eps/config) */
    BH_ERR_TOO_LARGE = -2,      /* n exceeds the context's max_n, or a size limit */
    BH_ERR_NONFINITE = -3,      /* a particle coordinate or mass is NaN or infinite */
    BH_ERR_CAPACITY = -4,       /* a device work list overflowed (walk stack); result invalid */
    BH_ERR_DEVICE_TIMEOUT = -5, /* a bounded device wait gave up; result invalid */
    BH_ERR_CUDA = -6,           /* a CUDA runtime call failed */
    BH_ERR_STATE = -7,          /* call order violated (e.g. tree_force before tree_build) */
    BH_ERR_NOMEM = -8           /* device allocation failed */
};

typedef struct bh_ctx bh_ctx;

/* Tunable parameters of one context (bh_config_default fills the defaults). */
typedef struct bh_config {
    int leaf_size;           /* n_leaf: a cell with <= n_leaf particles is a leaf (Sec. 4.1
                                splits down to one particle; n_leaf = 1 is the paper's tree) */
    int group_size;          /* G: particles per walk group, 1..256 */
    int order;               /* 1 = monopole (the paper), 2 = monopole + quadrupole */
    int fp64_node_threshold; /* nodes holding >= this many particles combine moments in FP64 */
    int block_threads;       /* threads per block of the walk kernel: 64 or 128 */
    int blocks_per_sm;       /* resident walk blocks per SM for the persistent grid (0 = auto) */
    int max_systems;         /* independent systems one bh_force_batched call may hold (>= 1) */
    int curve;               /* particle order (Sec. 5): BH_CURVE_MORTON (default) or
                                BH_CURVE_HILBERT (Peano-Hilbert); the octree is the same,
                                only the order of children and particles differs */
    int max_level;           /* deepest tree level: 10 (30-bit keys, default) or 21 (63-bit
                                keys, uint64 in BH_EXPORT_KEYS); deeper levels split the
                                dense cells that 10 levels leave as oversized leaves */
    int walk_variant;        /* tree_force kernel: BH_WALK_ONE_WARP (default: each warp walks
                                its group and evaluates the tiles it builds) or
                                BH_WALK_PAIRED (warp pairs: one walks and builds tiles, one
                                evaluates them; same tiles in the same order, so the same
                                bits).  The paired kernel serves G <= 96 with the plain
                                criterion, in blocks of 256 threads sized by occupancy
                                (block_threads and blocks_per_sm do not apply to it);
                                other cases take the one-warp kernel.
                                BH_WALK_TMA: the one-warp walk with its node records
                                and leaf particles staged into shared memory by bulk
                                asynchronous copies (cp.async.bulk), the next batch of
                                node records copied while the current tiles are
                                evaluated; same tiles in the same order, so the same
                                bits as BH_WALK_ONE_WARP.  With the learned criterion
                                the one-warp kernel runs */
} bh_config;

enum { BH_WALK_ONE_WARP = 0, BH_WALK_PAIRED = 1, BH_WALK_TMA = 2 };

#define BH_CURVE_MORTON 0
#define BH_CURVE_HILBERT 1

/* Counters of the last evaluation (bh_stats synchronises the stream). */
typedef struct bh_stats_t {
    int64_t n;               /* particles of the last tree_build */
    int64_t n_nodes;         /* tree nodes */
    int64_t n_leaves;        /* leaf nodes */
    int64_t n_groups;        /* walk groups */
    int64_t n_pp;            /* particle-particle interactions of the last tree_force (self excluded) */
    int64_t n_pc;            /* particle-cell interactions of the last tree_force */
    int64_t max_leaf_count;  /* largest leaf (only level-10 leaves may exceed leaf_size) */
    int32_t status;          /* device status word as a BH_* code */
    int32_t reserved;
    float box[4];            /* root cube: xmin, ymin, zmin, side L (Sec. 4.1) */
    int64_t n_pp_total;      /* particle-particle interactions since bh_create */
    int64_t n_pc_total;      /* particle-cell interactions since bh_create */
    int64_t launches;        /* kernels this context has enqueued since bh_create */
} bh_stats_t;

/* Library version (major * 10000 + minor * 100 + patch). */
int bh_version(void);

/* Human-readable name of a BH_* code (static string, never NULL). */
const char* bh_strerror(int code);

/* Fill *cfg with the defaults: leaf 8, group 64, order 1, FP64 threshold
 * 4096, 128 walk threads per block, automatic blocks per SM. */
void bh_config_default(bh_config* cfg);

/* Create a context on `device` for up to max_n particles (1 <= max_n < 2^30).
 * Allocates all device workspace up front (about 200 bytes per particle);
 * later calls allocate nothing.  cfg may be NULL (defaults).
 * Errors: BH_ERR_INVALID (bad cfg), BH_ERR_TOO_LARGE, BH_ERR_NOMEM, BH_ERR_CUDA. */
int bh_create(bh_ctx** out, const bh_config* cfg, int64_t max_n, int device);

/* Free a context and its workspace (NULL is ignored).  Synchronises its device. */
void bh_destroy(bh_ctx* ctx);

/* Steps 1-3 of the paper's flow (Sec. 4.4), on the device: the root cube
 * (Sec. 4.1), 30-bit Morton keys and a stable radix sort of the particles
 * into Morton order (Sec. 5), the octree (Sec. 4.1; leaf: <= leaf_size
 * particles or level 10) and the walk groups.
 * d_pos_mass: n float4 (x, y, z, m), read only by the work this call
 * enqueues; the context keeps its own Morton-ordered copy, so the buffer may
 * be reused once that work has run (stream order).
 * n = 0 is allowed (tree_force then writes nothing).
 * Errors: BH_ERR_INVALID, BH_ERR_TOO_LARGE (n > max_n); device status
 * BH_ERR_NONFINITE for a NaN/Inf coordinate or mass. */
int tree_build(bh_ctx* ctx, const float* d_pos_mass, int64_t n, void* stream);

/* Step 2 of Sec. 4.4: per node the total mass and centre of mass, the
 * quadrupole second moment when the context's order is 2, and Eq. (2)'s
 * effective size S_eff = (l/theta + s)^2 (l = cube side, s = distance from
 * the cube centre to the centre of mass).  theta > 0.
 * Errors: BH_ERR_INVALID (theta <= 0 or not finite), BH_ERR_STATE (no tree). */
int tree_moments(bh_ctx* ctx, float theta, void* stream);

/* Step 5 of Sec. 4.4: the tree walk and force evaluation.  Each group of
 * particles walks the tree once; a node is accepted when the squared
 * distance from its centre of mass to the group's bounding box exceeds
 * S_eff and it holds no group member (Eq. 2 applied to the whole group),
 * giving a particle-cell term; a rejected leaf gives particle-particle
 * terms (the target itself excluded); other rejected nodes are opened.
 * Interactions are FP32 with Kahan-compensated accumulation.
 * eps >= 0 is the Plummer softening of Eq. (1), applied to both kinds of term.
 * d_acc_pot: n float4 (ax, ay, az, phi) written in the caller's order.
 * Errors: BH_ERR_INVALID, BH_ERR_STATE (tree_moments not run after the last
 * tree_build); device status BH_ERR_CAPACITY or BH_ERR_DEVICE_TIMEOUT. */
int tree_force(bh_ctx* ctx, float eps, float* d_acc_pot, void* stream);

/* The paper's own walk (Sec. 4.4, Fig. 5, Appendix A): one thread per
 * particle follows the depth-first "more" (first child) and "next" (node
 * after the subtree) links from the root, with no stack.  For particle i a
 * node holding a single particle is a particle-particle term (skipped if it
 * is i); otherwise the node is accepted when |x_i - COM|^2 > S_eff (Eq. 2) and
 * it does not hold i, giving a particle-cell term (quadrupole when the
 * context's order is 2); a rejected leaf gives particle-particle terms with
 * its other members; a rejected internal node is entered.  The links are
 * derived from the current tree on each call.  FP32 terms, Kahan-compensated
 * runs of 32.  bh_stats then counts this walk's interactions.
 * eps >= 0: softening of Eq. (1).  flags: BH_PWALK_UNSOFTENED_CELLS applies
 * particle-cell terms with eps = 0, as the Appendix A kernel does;
 * BH_PWALK_INDIVIDUAL_SOFTENING uses the per-particle softening lengths set by
 * tree_softening (the symmetrized potential below; eps is then not used).
 * d_acc_pot: n float4 (ax, ay, az, phi) in the caller's order.
 * Errors: BH_ERR_INVALID, BH_ERR_STATE (tree_moments not run after the last
 * tree_build, or individual softening requested without tree_softening after
 * it); device status BH_ERR_CAPACITY for a malformed tree. */
#define BH_PWALK_UNSOFTENED_CELLS 1
#define BH_PWALK_INDIVIDUAL_SOFTENING 2
int tree_force_particles(bh_ctx* ctx, float eps, int flags, float* d_acc_pot, void* stream);

/* Individual softening with the symmetrized Plummer potential, the
 * application Sec. 7 names (after Saitoh & Makino 2010): particle i has its
 * own softening length eps_i; a pair (i, j) softens with
 * eps_ij^2 = (eps_i^2 + eps_j^2) / 2, so both bodies feel the same pair force
 * and momentum is conserved; a cell softens with (eps_i^2 + <eps^2>) / 2,
 * <eps^2> the mass-weighted mean over its particles (which cancels the term
 * of first order in the spread of eps^2, as the centre of mass cancels the
 * dipole; a massless cell takes 0).
 * Sets the softening of the particles of the tree of the last tree_build
 * (any later tree_build clears it) for tree_force_particles with
 * BH_PWALK_INDIVIDUAL_SOFTENING: d_eps holds n floats in the caller's order.
 * The first call on a context allocates its work arrays (cudaMalloc: 4 bytes
 * per particle and 20 per node of capacity), so it should come before any
 * stream capture; later calls allocate nothing.
 * Errors: BH_ERR_INVALID (bad pointer), BH_ERR_STATE (no tree), BH_ERR_NOMEM;
 * device status BH_ERR_NONFINITE for an eps that is negative or not finite. */
int tree_softening(bh_ctx* ctx, const float* d_eps, void* stream);

/* Neighbour search and SPH density, the short-range application of the
 * general tree walk (Sec. 4.3, Fig. 4), on the tree of the last tree_build
 * (tree_moments is not needed).  For particle i with search radius h_i,
 * j != i is a neighbour when |x_j - x_i| < h_i, decided in FP32 as
 * d = x_j - x_i per axis, r2 = fma(dz, dz, fma(dy, dy, dx * dx)), r2 < h_i * h_i.
 * rho_i = sum over i itself and its neighbours of m_j W(sqrt(r2), h_i), with
 * the cubic spline of Monaghan & Lattanzio (1985) of support h (unit
 * integral), FP32.  One warp walks the tree per particle group; a node is
 * skipped when its particles' bounding box is farther than the group's
 * largest radius from the group's box, so no neighbour is ever missed.
 * d_h: n radii in the caller's order, or NULL to use h for every particle.
 * d_count: n int32 neighbour counts (caller order, self excluded), or NULL.
 * d_rho: n float densities (caller order), or NULL.
 * bh_stats afterwards: n_pp = candidate pairs tested, n_pc = 0.
 * Errors: BH_ERR_INVALID (bad pointer, h <= 0 or not finite with d_h NULL),
 * BH_ERR_STATE (no tree); device status BH_ERR_NONFINITE for a radius that
 * is not positive and finite, BH_ERR_CAPACITY. */
int tree_neighbors(bh_ctx* ctx, const float* d_h, float h, int32_t* d_count, float* d_rho, void* stream);

/* Eq. (1) by direct summation (Sec. 3): for each target t,
 * a_t = sum_j m_j (x_j - x_t) / (|x_j - x_t|^2 + eps^2)^1.5 and
 * phi_t = -sum_j m_j / (|x_j - x_t|^2 + eps^2)^0.5 over all sources j except
 * d_tgt_self[t] (an index into the sources, or -1; d_tgt_self may be NULL).
 * d_src: n_src float4 (x, y, z, m); d_tgt: n_tgt float4 (x, y, z, ignored).
 * precision 32: FP32 interactions, Kahan-compensated, d_out = n_tgt float4;
 * precision 64: FP64 throughout, d_out = n_tgt double4 (the error judge).
 * No context is needed; nothing is allocated.
 * Errors: BH_ERR_INVALID (bad pointer/alignment/precision, eps < 0),
 * BH_ERR_TOO_LARGE (n_src or n_tgt >= 2^31). */
int direct_force(const float* d_src, int64_t n_src, const float* d_tgt, const int64_t* d_tgt_self,
                 int64_t n_tgt, double eps, void* d_out, int precision, void* stream);

/* direct_force with individual softening lengths and the symmetrized
 * Plummer potential (Sec. 7, after Saitoh & Makino 2010): the pair (t, j)
 * softens with (eps_t^2 + eps_j^2) / 2.  d_eps_src: n_src floats (one per
 * source), d_eps_tgt: n_tgt floats (one per target); the rest as
 * direct_force (precision 64 is the error judge of the symmetrized walk).
 * Errors: as direct_force. */
int direct_force_sym(const float* d_src, const float* d_eps_src, int64_t n_src, const float* d_tgt,
                     const float* d_eps_tgt, const int64_t* d_tgt_self, int64_t n_tgt, void* d_out, int precision,
                     void* stream);

/* The orbit loop of Sec. 1 ("compute forces, integrate, repeat"): one
 * leapfrog update per particle, v += a * dt_kick then x += v * dt_drift.
 * A kick-drift-kick step is bh_kick_drift(dt/2 then dt) after the first
 * force, then force, then the next call's dt/2 kick (or dt_kick = dt when the
 * two half kicks are merged).
 * d_pos: n float4 (x, y, z, m), positions updated in place, m untouched;
 * d_vel: n float4 (vx, vy, vz, unused), updated in place;
 * d_acc: n float4 (ax, ay, az, phi) from tree_force (caller order).
 * Errors: BH_ERR_INVALID (null/misaligned/non-device pointer, n < 0). */
int bh_kick_drift(bh_ctx* ctx, float* d_pos, float* d_vel, const float* d_acc, int64_t n, float dt_kick,
                  float dt_drift, void* stream);

/* ---------------------------------------------------------------------------
 * Many independent systems in one evaluation (the paper evaluates one system;
 * this batches the same method).  Each system gets its own root cube, Morton
 * order and tree; all systems are built by the same few launches and walked
 * by one persistent walk launch whose work queue holds every system's groups.
 * ------------------------------------------------------------------------- */

/* Fix the layout of the next bh_force_batched calls: h_offsets (host, nsys+1
 * int64) = first particle of each system, h_offsets[0] = 0, nondecreasing;
 * each system holds at most 65536 particles; the total at most max_n;
 * 1 <= nsys <= cfg.max_systems.  Synchronous (copies the layout to the
 * device); call it outside any stream capture.
 * Errors: BH_ERR_INVALID, BH_ERR_TOO_LARGE. */
int bh_batch_layout(bh_ctx* ctx, const int64_t* h_offsets, int nsys);

/* Forces of every system of the layout: d_pos_mass holds the systems'
 * particles back to back (float4 x, y, z, m), d_acc_pot receives
 * (ax, ay, az, phi) in the same order; systems never interact.  Same method
 * as tree_build + tree_moments(theta) + tree_force(eps) per system (plain
 * Eq. 2 criterion).  Stream-ordered, allocates nothing, syncs nothing: it can
 * be captured in a CUDA graph (see bh_graph_capture_batched).
 * Errors: BH_ERR_INVALID, BH_ERR_STATE (no layout, or the learned criterion is on). */
int bh_force_batched(bh_ctx* ctx, const float* d_pos_mass, float theta, float eps, float* d_acc_pot, void* stream);

/* Capture one bh_force_batched call into an executable CUDA graph
 * (*graph_exec, a cudaGraphExec_t passed as void*); replay it with
 * bh_graph_launch on any stream, free it with bh_graph_destroy.  The graph
 * keeps the pointers and parameters given here.
 * Errors: those of bh_force_batched, BH_ERR_CUDA. */
int bh_graph_capture_batched(bh_ctx* ctx, const float* d_pos_mass, float theta, float eps, float* d_acc_pot,
                             void** graph_exec);
int bh_graph_launch(void* graph_exec, void* stream);
void bh_graph_destroy(void* graph_exec);

/* ---------------------------------------------------------------------------
 * Learned opening criterion.  An extension of Eq. (2)'s test (the paper's
 * criterion is purely geometric): a 6 -> 32 -> 32 -> 1 ReLU network predicts
 * log10 of a node's relative force-error contribution to a group from the
 * features f1 = l/d (l cube side, d = |COM - group box centre|),
 * f2 = log10(M/M_total), f3 = |I - (T/3)1|_F / (M l^2) (0 for order 1),
 * f4 = r_g/d (r_g = half diagonal of the group box), f5 = level/10,
 * f6 = log2(count)/24.  Parameters: 1313 floats packed W1[32][6], b1[32],
 * W2[32][32], b2[32], W3[32], b3.  In the walk the network runs as BF16
 * tensor-core MMAs with FP32 accumulation.
 * ------------------------------------------------------------------------- */

/* Switch ctx to the learned criterion (h_params: host, 1313 FP32) or back to
 * the plain criterion (h_params NULL).  With the learned criterion a node is
 * accepted when Eq. (2) with the theta given to tree_moments (the guard)
 * passes, it holds no group member, and the prediction is below log10(tau);
 * if a feature lies outside [h_fmin[k], h_fmax[k]] (host, 6 floats each) the
 * plain criterion at theta_fb decides instead.  Synchronises the device;
 * tree_moments must run again before tree_force.
 * Errors: BH_ERR_INVALID (tau or theta_fb <= 0, non-finite parameters). */
int bh_mac_set(bh_ctx* ctx, const float* h_params, const float* h_fmin, const float* h_fmax, float tau,
               float theta_fb);

/* Training data for the criterion, measured by the method itself: for each
 * group index in d_groups (n_groups int32) the kernel walks the tree with the
 * guard (Eq. 2 at tree_moments' theta, no member held) and, for every node
 * passing it, writes the six features to d_X (float[cap][6]) and the label
 * log10(max over members of |a_PC(node) - a_direct(node)| / |a_ref|) to d_Y
 * (float[cap]); a_direct sums the node's particles, d_acc_ref (n float4,
 * caller order) gives each member's reference total acceleration.  It also
 * descends into such nodes while their label exceeds log10_floor.
 * *d_count (device u64, caller-zeroed) receives the number of pairs found;
 * only the first cap are written, in no particular order; d_pairs (int32
 * [cap][2], or NULL) receives each pair's (node index, group index).
 * Needs tree_build + tree_moments.
 * Errors: BH_ERR_INVALID, BH_ERR_STATE. */
int bh_mac_label(bh_ctx* ctx, const int32_t* d_groups, int64_t n_groups, const float* d_acc_ref, float eps,
                 float log10_floor, float* d_X, float* d_Y, int32_t* d_pairs, int64_t cap,
                 unsigned long long* d_count, void* stream);

/* `steps` Adam steps (lr, beta 0.9 / 0.999, eps 1e-8; step t0+1 onwards) of
 * the network on (d_X float[n][6], d_Y float[n]) with the weighted squared
 * loss w (y_hat - y)^2, w = under_weight when y_hat < y (an under-estimated
 * error is the unsafe side) else 1.  Mini-batches of `batch` samples are
 * taken in the order d_order (int32[n], a permutation drawn by the caller;
 * NULL = 0..n-1), continuing from sample t0*batch.  d_params (1313 FP32
 * master weights), d_adam_m / d_adam_v (1313 each) are updated in place;
 * d_loss (float[steps], caller-zeroed, or NULL) receives each step's loss.
 * d_work: at least batch*135 + 1313 floats of scratch.
 * Errors: BH_ERR_INVALID, BH_ERR_TOO_LARGE (work too small). */
int bh_mlp_train(const float* d_X, const float* d_Y, const int32_t* d_order, int64_t n, float* d_params,
                 float* d_adam_m, float* d_adam_v, float* d_work, int64_t work_floats, int64_t steps, int batch,
                 float lr, float under_weight, float* d_loss, int64_t t0, void* stream);

/* Gradient (d_grad, 1313) and loss (*d_loss, caller-zeroed, or NULL) of the
 * mean weighted loss over n samples, FP32.  d_work: n*135 floats.
 * Errors: BH_ERR_INVALID, BH_ERR_TOO_LARGE. */
int bh_mlp_grad(const float* d_params, const float* d_X, const float* d_Y, int64_t n, float under_weight,
                float* d_work, int64_t work_floats, float* d_grad, float* d_loss, void* stream);

/* Network predictions d_y[n] for d_X[n][6]: precision 32 = FP32 with the
 * device parameters d_params (training path); precision 16 = the walk's BF16
 * tensor-core path with the network loaded into ctx by bh_mac_set.
 * Errors: BH_ERR_INVALID, BH_ERR_STATE (precision 16 without a network). */
int bh_mlp_forward(bh_ctx* ctx, const float* d_params, const float* d_X, int64_t n, float* d_y, int precision,
                   void* stream);

/* Whole force evaluation for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a service of this library.  Code
 * that runs while a CUDA graph is being captured (cudaMalloc is illegal
 * there), plugins whose host application owns all device memory, and
 * real-time loops that must never allocate cannot use bh_create's slab.
 * This entry point runs the same kernels as tree_build + tree_moments +
 * tree_force, with its work arrays in a fixed file-scope device array of
 * BH_STATIC_SCRATCH_BYTES (16 MiB), which every GPU that loads the library
 * holds until the process exits; it calls no allocating routine.
 * Limits: n <= BH_STATIC_MAX_N (32768), and the work arrays of (n, cfg)
 * must fit in the array (true for leaf_size >= 4 at n = 32768); larger
 * requests return BH_ERR_TOO_LARGE.
 * The first call on each device (with that device current) looks up the
 * array's device address and clears it, synchronously: make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents, so calls that overlap on the GPU (two streams, two
 * host threads on one device) race; serialise them.
 * d_pos_mass: n float4 (x, y, z, m); d_acc_pot: n float4 (ax, ay, az, phi),
 * caller order; cfg may be NULL (defaults); theta > 0, eps >= 0.
 * h_status: NULL, or a host int that receives the device status (BH_OK or a
 * BH_ERR_* code) after the call synchronises `stream`.
 * Errors: BH_ERR_INVALID, BH_ERR_TOO_LARGE, BH_ERR_CUDA. */
#define BH_STATIC_SCRATCH_BYTES (16u << 20)
#define BH_STATIC_MAX_N 32768
int bh_tree_force_static(const float* d_pos_mass, int64_t n, const bh_config* cfg, float theta, float eps,
                         float* d_acc_pot, int* h_status, void* stream);

/* Failure-path self-test: launches one bounded device wait that nothing
 * will satisfy, of the kind the library's kernels use, so that a deployment
 * can check that such a wait ends and is reported.
 *   which = BH_SELFTEST_TILE_RING: the paired walk's mbarrier wait (gives up
 *           after one second of %globaltimer time or 2^22 polls, whichever
 *           comes first);
 *   which = BH_SELFTEST_LOOKBACK:  the sort's decoupled look-back wait
 *           (gives up after 2^22 polls, well under a second);
 *   which = BH_SELFTEST_TMA:       the TMA-staged walk's wait for its bulk
 *           copies, on an mbarrier told to expect 16 bytes that no copy
 *           delivers (gives up like the tile ring's wait).
 * Asynchronous on `stream`; afterwards bh_status returns
 * BH_ERR_DEVICE_TIMEOUT (and clears it) and the context stays usable.
 * Errors: BH_ERR_INVALID (null context, unknown `which`), BH_ERR_CUDA. */
enum { BH_SELFTEST_TILE_RING = 0, BH_SELFTEST_LOOKBACK = 1, BH_SELFTEST_TMA = 2 };
int bh_selftest_wait(bh_ctx* ctx, int which, void* stream);

/* Synchronise `stream` and return the context's device status as a BH_*
 * code (BH_OK if no device-side error was recorded since the last call;
 * the status is then cleared). */
int bh_status(bh_ctx* ctx, void* stream);

/* Synchronise `stream`, then report counters of the last build/evaluation
 * and the status word (not cleared). */
int bh_stats(bh_ctx* ctx, void* stream, bh_stats_t* out);

/* Copy an internal array of the last build into caller memory (device or
 * host: the copy direction is inferred), for inspection and tests.
 * what: BH_EXPORT_* below; cap_bytes: capacity of dst.  *out_bytes receives
 * the byte count of the array.  Stream-ordered; synchronises the stream to
 * read the array's current length.
 * Errors: BH_ERR_INVALID, BH_ERR_TOO_LARGE (cap_bytes too small), BH_ERR_STATE. */
enum {
    BH_EXPORT_KEYS = 1,        /* uint32[n]   sorted keys (uint64[n] when max_level = 21) */
    BH_EXPORT_PERM = 2,        /* uint32[n]   caller index of each Morton-ordered particle */
    BH_EXPORT_SPOS = 3,        /* float4[n]   particles in Morton order */
    BH_EXPORT_NODE_FIRST = 4,  /* int32[nn]   first particle (Morton position) of each node */
    BH_EXPORT_NODE_COUNT = 5,  /* int32[nn]   particle count of each node */
    BH_EXPORT_NODE_CHILD = 6,  /* int32[nn]   index of the first child, -1 for leaves */
    BH_EXPORT_NODE_NCHILD = 7, /* int32[nn]   number of children (0 for leaves) */
    BH_EXPORT_NODE_LEVEL = 8,  /* int32[nn]   level (0 = root cube) */
    BH_EXPORT_COM_M = 9,       /* float4[nn]  centre of mass and mass */
    BH_EXPORT_SEFF = 10,       /* float[nn]   S_eff of Eq. (2) */
    BH_EXPORT_QUAD = 11,       /* float[nn*6] second moments xx, yy, zz, xy, xz, yz (order 2) */
    BH_EXPORT_GROUP_FIRST = 12,/* int32[ng]   first particle of each group */
    BH_EXPORT_GROUP_COUNT = 13,/* int32[ng]   particles per group */
    BH_EXPORT_BOX = 14,        /* float[4]    xmin, ymin, zmin, L */
    BH_EXPORT_NEXT = 15        /* int32[nn]   depth-first "next" link of each node, -1 after the last
                                  (derived by tree_force_particles; Fig. 5) */
};
int bh_export(bh_ctx* ctx, int what, void* dst, int64_t cap_bytes, int64_t* out_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BHTREE_H */
