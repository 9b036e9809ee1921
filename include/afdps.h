/*
 * afdps.h -- C ABI of the GB300 (sm_103a) multiwalk, indirect-index
 * Barnes-Hut gravity library (method of "Accelerated FDPS", Iwasawa et al.,
 * arXiv 1907.02290).
 *
 * The library computes softened gravitational accelerations and potentials
 * with the tree method: Morton-key octree (Section 4.3), i-groups of at most
 * n_grp particles sharing one interaction list (Barnes' vectorisation,
 * Section 2), many groups per kernel launch (multiwalk, Section 3), lists of
 * particle and superparticle INDICES into device-resident arrays (indirect
 * addressing, Section 4.1), and lists kept and reused across steps while the
 * moments are recomputed (list reuse, Section 4.2). The three list modes
 * mirror the paper's MAKE_LIST / MAKE_LIST_FOR_REUSE / REUSE_LIST (Section 5).
 *
 * Conventions shared by every entry point:
 *  - Particle arrays are device pointers to FP64 structure-of-arrays data in
 *    the caller's particle order (x, y, z, m: one double per particle). The
 *    caller owns them; they must stay valid until the work queued by the call
 *    has run on the context's stream. Nothing is copied to the host unless the
 *    entry point says so.
 *  - Outputs (acc4) are device pointers, caller particle order: four floats
 *    per particle (ax, ay, az, phi), 16-byte aligned. G = 1.
 *  - Work is queued on the CUDA stream given at creation (or set later); the
 *    calls that build a tree or lists synchronise that stream once to size
 *    their buffers, the reuse step and the force calculation do not.
 *  - The context owns the tree, groups, lists and scratch memory (device
 *    allocations made with cudaMalloc, grown on demand, freed by
 *    afd_destroy).
 *  - Every int-returning call returns AFD_OK (0) or a negative afd_status;
 *    nothing throws across the ABI. Errors found by device code in calls that
 *    do not synchronise (non-finite input in a reuse step, a walk that ran
 *    out of stack) are kept in a device status word and returned by the next
 *    synchronising call or by afd_sync().
 *  - One context is not thread-safe; different contexts are independent.
 */
#ifndef AFDPS_H
#define AFDPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afd_ctx afd_ctx;

/* List modes of the top-level call (Section 5: the FDPS enum). */
typedef enum {
  AFD_MAKE_LIST = 0,           /* build tree + lists, do not keep them for reuse */
  AFD_MAKE_LIST_FOR_REUSE = 1, /* build tree + lists and keep them */
  AFD_REUSE_LIST = 2           /* keep topology and lists; recompute moments */
} afd_list_mode;

typedef enum {
  AFD_OK = 0,
  AFD_ERR_ARG = -1,           /* bad argument (null pointer, bad config, n < 0) */
  AFD_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  AFD_ERR_NONFINITE = -3,     /* a coordinate or mass is NaN or infinite */
  AFD_ERR_NO_SAVED_LIST = -4, /* REUSE_LIST without lists made for reuse */
  AFD_ERR_SHAPE = -5,         /* particle count differs from the saved tree */
  AFD_ERR_LIST_OVERFLOW = -6, /* a list or cell count exceeds 32-bit indexing */
  AFD_ERR_TIMEOUT = -7,       /* a bounded device wait gave up */
  AFD_ERR_NO_TREE = -8,       /* lists or force requested before a tree */
  AFD_ERR_OOM = -9,           /* device allocation failed */
  AFD_ERR_WALK_STACK = -10,   /* a tree walk overflowed its per-warp stack */
  AFD_ERR_TOO_LARGE = -11,    /* problem size above the limit of afd_root_cell_static */
  AFD_ERR_NO_REFERENCE = -12, /* learned-criterion sampling without reference accelerations */
  AFD_ERR_BAD_RADIUS = -13    /* a search radius is not finite and positive */
} afd_status;

/* Method parameters. Paper values: n_leaf = 16, theta in [0.25, 1]
 * (Section 6.1); eps and the multipole order are not given by the paper. */
typedef struct {
  double eps;            /* Plummer softening length, >= 0 */
  double theta;          /* opening angle, >= 0 (0 opens every cell) */
  int32_t n_leaf;        /* a cell splits while it holds more particles, >= 1 */
  int32_t n_grp;         /* maximum particles per i-group, 1 .. 1024 */
  int32_t multipole;     /* 0: monopole superparticles, 1: + quadrupole */
  int32_t far_precision; /* 0: FP32 superparticle terms, 1: BF16, 2: FP16 */
  int32_t mac;           /* 0: theta criterion; 1: learned criterion allowed (see
                            afd_mac_set; quadrupole moments are then always kept) */
  int32_t reserved;      /* must be 0 */
} afd_config;

/* Create a context on CUDA device `device`, queuing work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream). *out receives the
 * context. Returns AFD_ERR_ARG for a bad config. */
int afd_create(afd_ctx **out, const afd_config *cfg, int device, void *stream);

/* Free every device buffer of the context (synchronises its stream). */
void afd_destroy(afd_ctx *ctx);

/* Several independent systems in one context (the batched multiwalk: every
 * kernel, the force kernel included, runs once over all systems). Particles
 * [sys_off[s], sys_off[s+1]) of the arrays later given to afd_tree_build form
 * system s, with its own root cell, keys, tree and groups; lists never cross
 * systems. sys_off: host, n_sys + 1 non-decreasing offsets from 0. n_grp:
 * host, n_sys group sizes (1 .. 1024), or NULL for the config's n_grp.
 * n_sys = 1 with sys_off = {0, n} is the single-system default. Invalidates
 * the tree and lists. Synchronous. */
int afd_set_systems(afd_ctx *ctx, const int64_t *sys_off, int n_sys, const int32_t *n_grp);

/* Replace the stream later work is queued on. */
int afd_set_stream(afd_ctx *ctx, void *stream);

/* Tree construction (Section 4.3): root cell from all positions, 63-bit
 * Morton keys (21 bits per axis), stable LSD radix sort of (key, index),
 * reorder of the particle data into Morton order, level-wise octree link,
 * bottom-up monopole (and quadrupole) moments, and i-groups. x, y, z, m are
 * n device doubles each (caller order), 0 <= n < 2^30 (n = 0 gives an empty
 * tree).
 * Synchronises once. Invalidates saved lists. AFD_ERR_NONFINITE if a
 * coordinate or mass is not finite, or if a system's extent has no finite
 * power-of-two side (1.000001 x the extent above 2^1023). */
int afd_tree_build(afd_ctx *ctx, const double *x, const double *y, const double *z,
                   const double *m, int64_t n);

/* Interaction lists for every i-group (Sections 2, 3, 4.1): a depth-first
 * walk under the opening-angle criterion producing, per group, a list of
 * particle indices (EPJ) and a list of cell indices (SPJ) into the device
 * arrays. mode is AFD_MAKE_LIST or AFD_MAKE_LIST_FOR_REUSE; the latter keeps
 * the lists for later AFD_REUSE_LIST steps. Also orders the force kernel's
 * work items by list work, longest first (a launch order only: the forces do
 * not depend on it). Needs a tree. Synchronises once. */
int afd_make_interaction_lists(afd_ctx *ctx, int mode);

/* Reusing step (Section 4.2): keep the topology, groups and lists; reorder
 * the new particle data with the saved permutation and recompute the cell
 * moments bottom-up. x, y, z, m: device doubles, same n as the saved tree.
 * With neighbour lists kept but no interaction lists made for reuse, only
 * the particles are reordered (the density needs nothing else); the moments
 * are then recomputed by the next call that reads them (a list walk, the
 * local essential tree export, learned-criterion sampling). Interaction
 * lists made with AFD_MAKE_LIST end here. Does not synchronise.
 * AFD_ERR_NO_SAVED_LIST without interaction lists kept for reuse or
 * neighbour lists. */
int afd_reuse_lists(afd_ctx *ctx, const double *x, const double *y, const double *z,
                    const double *m);

/* Force kernel (Section 5, the indirect-index dispatch): for every group and
 * every EPJ / SPJ index of its list, sum the softened attraction on each of
 * the group's particles. One warp takes 32 of a group's particles, or up to
 * 64 (a full 32-particle unit and the group's next unit when that holds more
 * than 16 particles, monopole lists), in the launch order set by
 * afd_make_interaction_lists. acc4: device, n x (ax, ay, az,
 * phi) floats, caller order, overwritten. Does not synchronise.
 * The potential is the FP32 kernel's (compensated sums, rms relative
 * difference from an FP64 sum over the same lists about 1e-7, far below the
 * tree's own approximation error of 1e-4 .. 1e-3 at theta 0.3 .. 0.7); no
 * FP64 potential is written, since an FP64 copy of it would carry no more
 * correct digits. Energies are summed in FP64 by afd_energy. */
int afd_calc_force(afd_ctx *ctx, float *acc4);

/* The top-level call of Section 5 (calcForceAllAndWriteBackMultiWalkIndex):
 * MAKE_LIST / MAKE_LIST_FOR_REUSE build the tree and lists, REUSE_LIST runs
 * the reusing step; then the force kernel writes acc4. */
int afd_calc_force_all(afd_ctx *ctx, const double *x, const double *y, const double *z,
                       const double *m, int64_t n, float *acc4, int mode);

/* The same top-level call on HOST arrays (caller order): copies x, y, z, m
 * to the device, runs afd_calc_force_all, returns the n x 4 floats in
 * acc4_host and synchronises. Pinned host memory gives the fastest copies;
 * when acc4_host is pinned and mapped (cudaHostAlloc, or registered with a
 * device pointer) and neither the learned criterion nor a work share is
 * set, the force kernel writes it directly over the host link while it
 * runs, with no copy after it. The contents of acc4_host are undefined
 * while the call runs. */
int afd_calc_force_all_host(afd_ctx *ctx, const double *x, const double *y, const double *z,
                            const double *m, int64_t n, float *acc4_host, int mode);

/* Kick-drift (first half of a KDK leapfrog step, caller order, device
 * arrays): v += a * dt_kick, then x += v * dt_drift. acc4 as written by
 * afd_calc_force. */
int afd_kick_drift(afd_ctx *ctx, double *x, double *y, double *z, double *vx, double *vy,
                   double *vz, const float *acc4, int64_t n, double dt_kick, double dt_drift);

/* Kick: v += a * dt_kick. */
int afd_kick(afd_ctx *ctx, double *vx, double *vy, double *vz, const float *acc4, int64_t n,
             double dt_kick);

/* n_steps kick-drift-kick steps of size dt on device arrays. acc4 holds the
 * accelerations at the start and receives those at the end. Force
 * evaluation k of the context (counted since the last AFD_MAKE_LIST_FOR_REUSE
 * issued by this call) rebuilds the tree and lists when k % n_reuse == 0 and
 * reuses them otherwise; the first evaluation of a call always rebuilds. */
int afd_leapfrog(afd_ctx *ctx, double *x, double *y, double *z, double *vx, double *vy,
                 double *vz, const double *m, int64_t n, float *acc4, double dt, int n_steps,
                 int n_reuse);

/* FP64 energies: out[0] = sum m v^2 / 2, out[1] = sum m phi / 2 (phi from
 * acc4). Host array of two doubles; synchronises. */
int afd_energy(afd_ctx *ctx, const double *vx, const double *vy, const double *vz,
               const double *m, const float *acc4, int64_t n, double *out);

/* Per-system work of the current lists: inter[s] = interactions of system s
 * (sum over its groups of n_i (n_epj + n_spj)), entries[s] = its list
 * entries. Host arrays of n_sys int64. Synchronises. */
int afd_system_stats(afd_ctx *ctx, int64_t *inter, int64_t *entries);

/* Capture one reusing timestep into a CUDA graph owned by the context:
 * kick-drift (v += a dt/2, x += v dt), the reusing step of Section 4.2
 * (reorder with the saved permutation, moments), the force kernel on the
 * saved lists, kick. The arrays (device, caller order) must keep their
 * addresses for every replay; the context's stream must not be the legacy
 * default stream; lists must have been made for reuse. Nothing runs at
 * capture time, and work already queued on the stream keeps running (the
 * call waits only for a replay of the context's previous graph); a replay
 * is ordered after it on the stream. Replay with afd_graph_launch; a new
 * construction step (afd_tree_build with more cells or groups) requires a
 * new capture. */
int afd_graph_capture_step(afd_ctx *ctx, double *x, double *y, double *z, double *vx,
                           double *vy, double *vz, const double *m, float *acc4, double dt);

/* Replay the captured timestep on the context's stream (one launch). */
int afd_graph_launch(afd_ctx *ctx);

/* Autotune the group size n_grp -- the adjustable parameter of Barnes'
 * vectorisation and of the multiwalk (Sections 3 and 6.1) -- for the
 * particles x, y, z, m (device, n, the systems set by afd_set_systems). For
 * each candidate cand[0..n_cand) (1 .. 1024) the tree, the lists and the
 * force are computed twice and timed with CUDA events on the second pass;
 * each system gets the candidate minimising t_construction * (its share of
 * list entries) / n_reuse + t_force * (its share of interactions). The
 * choice is written to best (host, n_sys ints) and installed as the group
 * sizes (via afd_set_systems, or the config's n_grp for one system). acc4
 * (device, n x 4 floats) is scratch. Synchronises; leaves no tree. */
int afd_autotune_n_grp(afd_ctx *ctx, const double *x, const double *y, const double *z,
                       const double *m, int64_t n, const int32_t *cand, int n_cand, int n_reuse,
                       float *acc4, int32_t *best);

/* Launch shape of the force kernel: warps per block (2, 4 or 8) and list
 * entries staged per chunk by each warp (32 or 64). Defaults 4 and 32. The
 * results do not depend on it beyond FP32 summation order within a chunk. */
int afd_set_launch(afd_ctx *ctx, int warps_per_block, int chunk);
int afd_get_launch(afd_ctx *ctx, int *warps_per_block, int *chunk);

/* Autotune the force kernel's launch shape on the current lists: every
 * (chunk, warps) in {32, 64} x {2, 4, 8} is launched once to warm up, then
 * timed over `reps` launches with CUDA events on the context's stream; the
 * fastest is installed. ms_out (host, 6 floats, may be NULL) receives the
 * mean ms per launch, index chunk_index * 3 + warps_index. acc4 (device,
 * n x 4 floats) receives the forces. Needs lists; synchronises. */
int afd_autotune_launch(afd_ctx *ctx, float *acc4, int reps, float *ms_out);

/* The non-indirect ablation of the force calculation (the paper compares
 * the indirect scheme with sending each group's j-data itself, Section 4.1):
 * copy the j-data (hi/lo float4 pairs) of every EPJ and SPJ list entry into
 * list order (device buffers owned by the context, 32 bytes per entry), then
 * run the same force kernel reading those copies contiguously instead of by
 * index. The forces equal afd_calc_force's bit for bit. Monopole lists only
 * (AFD_ERR_ARG with quadrupoles). ms_out (host, 2 floats, may be NULL): the
 * copy and the force kernel, CUDA-event milliseconds. Synchronises. */
int afd_calc_force_materialized(afd_ctx *ctx, float *acc4, float *ms_out);

/* Local essential tree of the current tree for a remote domain (Section 3;
 * Section 4.3: the global tree is built over the local particles and the
 * superparticles and particles imported from other domains). box (host, 6
 * doubles: min x y z, max x y z) is the remote domain; the export is what
 * the interaction-list walk with that box as the group box and opening
 * angle theta puts on a list: each accepted cell as one superparticle (its
 * FP64 COM and monopole), each opened leaf as its particles, in depth-first
 * order (children in Morton order). The first min(total, cap) elements go to
 * x, y, z, m (device doubles, cap each) and kind (device u32, 0 particle,
 * 1 superparticle; may be NULL); *n_out (host) = total. A receiving
 * context builds its tree over its own particles followed by the imported
 * elements (afd_tree_build) and keeps the forces of its own particles.
 * Monopole superparticles; one system per context (AFD_ERR_ARG otherwise);
 * needs a tree. Synchronises. */
int afd_let_export(afd_ctx *ctx, const double *box, double theta, int64_t cap, double *x,
                   double *y, double *z, double *m, uint32_t *kind, int64_t *n_out);

/* ---------------------------------------------------------------------------
 * Short-range neighbour walk (Section 2: short-range interactions such as
 * SPH use the same tree walk with a cell-opening criterion other than the
 * opening angle; Section 4.2: their lists can be kept over several steps,
 * since particles move a small fraction of their spacing per step).
 * ------------------------------------------------------------------------- */

/* Neighbour lists of the current tree, one per i-group, for the search
 * radii h (device, n doubles, caller order, each finite and > 0) and the
 * margin skin (host double, finite, >= 0). The search box of a group is,
 * per axis, [min_i (x_i - (h_i + skin)), max_i (x_i + (h_i + skin))] over
 * its particles, each bound computed in FP64 and rounded outward to FP32;
 * the tight box of a cell is the min / max of its particles' coordinates
 * rounded outward to FP32. A cell whose tight box meets the search box is
 * opened (or listed, when a leaf); any other cell is dropped with its
 * subtree. A group's list is the particles of its listed leaves in
 * depth-first order, which is ascending Morton position: every particle
 * within h_i + skin of a particle i is on the list of i's group. Lists
 * stay in the context until the next afd_tree_build and are kept by
 * afd_reuse_lists (moves of less than skin / 2 keep every neighbour within
 * h_i). Independent systems (afd_set_systems) get lists of their own
 * particles. Needs a tree; synchronises. AFD_ERR_BAD_RADIUS if a radius is
 * not finite and positive, AFD_ERR_ARG for a bad skin. */
int afd_make_neighbour_lists(afd_ctx *ctx, const double *h, double skin);

/* Gather-form SPH density over the neighbour lists, with the current
 * positions and masses: rho_i = sum_j m_j W(|x_j - x_i|, h_i), the particle
 * itself included, W the M4 cubic spline of support radius h in three
 * dimensions, W(r, h) = 8 / (pi h^3) w(r / h) with w(q) = 1 - 6 q^2 + 6 q^3
 * for q <= 1/2, 2 (1 - q)^3 for 1/2 < q < 1 and 0 beyond; and the smooth
 * neighbour number nnb_i = (32 / 3) sum_j w(|x_j - x_i| / h_i). h (device,
 * n doubles, caller order) are this evaluation's radii; they may differ
 * from the lists' as long as every neighbour is still on the lists (h_i
 * below the list radius + skin - twice the largest move since the lists
 * were made). rho, nnb (device, n floats each, caller order; nnb may be
 * NULL). FP32 arithmetic on coordinates relative to the group's first
 * particle. Stream-ordered, does not synchronise; a radius that is not
 * finite and positive gives NaN there and AFD_ERR_BAD_RADIUS at the next
 * afd_sync. AFD_ERR_NO_SAVED_LIST without neighbour lists. */
int afd_calc_density(afd_ctx *ctx, const double *h, float *rho, float *nnb);

/* Sizes of the neighbour lists (host int64[2]): out[0] list entries,
 * out[1] candidate pairs of one density evaluation (sum over groups of
 * n_i x list length). Zeros without lists. */
int afd_neighbour_stats(afd_ctx *ctx, int64_t *out);

/* ---------------------------------------------------------------------------
 * A force step split over several processes (one GPU each) by disjoint
 * slices of i-groups: every process builds the same tree and lists, computes
 * the forces of its part of the groups, and the parts' outputs are combined
 * by the caller (zero-filled outputs summed, e.g. an all-reduce). The
 * groups' outputs are disjoint, so the combined forces equal an unshared
 * evaluation's bit for bit.
 * ------------------------------------------------------------------------- */

/* Contiguous, balanced parts of a work array (host memory, no GPU): bounds
 * (host, parts + 1 int64) receives bounds[0] = 0 <= bounds[1] <= ... <=
 * bounds[parts] = n, where bounds[p] is the first index whose prefix sum
 * work[0] + ... + work[k - 1] reaches total * p / parts; each part's work is
 * within one element's work of total / parts. All-zero work is split by
 * count. AFD_ERR_ARG for n < 0, parts < 1 or null pointers. */
int afd_partition_work(const uint64_t *work, int64_t n, int parts, int64_t *bounds);

/* Take part `part` of `parts` (0 <= part < parts) of every later force
 * evaluation: at each list construction the groups are split by
 * afd_partition_work over their work n_i x (EPJ + SPJ list length), and
 * afd_calc_force (and the steps that call it) writes the forces of this
 * part's groups only, leaving the other rows of acc4 untouched. parts = 1
 * (the default) computes everything. With the learned criterion the caller
 * passes the combined forces to afd_mac_set_reference. Synchronises when
 * lists exist (the split of the current lists is made at once). */
int afd_set_work_share(afd_ctx *ctx, int part, int parts);

/* The current share (host int64[5]): part, parts, first and end group of
 * this part's slice, and its interactions (sum of n_i x list length). */
int afd_get_work_share(afd_ctx *ctx, int64_t *out);

/* Limits of the tree walks' bounded device loops, for tests of the error
 * paths (the defaults never bind on valid input). iter_cap: warp steps a
 * walk may take for one group (or neighbour-walk item) before it stops and
 * the call returns AFD_ERR_TIMEOUT (default 2 x cells + 64, which a walk
 * never reaches: every step removes at least one stack entry or expands a
 * cell). stack_cap: stack entries per warp, 1 .. 448 (the shared-memory
 * stack); a walk that would need more stops with AFD_ERR_WALK_STACK
 * (default 448, above what a depth-21 tree can need). arena_chunks_max:
 * the largest record arena of the list construction, in chunks of 64
 * records, 1 .. 2^30 (default 2^30); lists that do not fit return
 * AFD_ERR_LIST_OVERFLOW. 0 restores a default. A walk that stops leaves
 * the context without lists and usable. Host only; no synchronisation.
 * AFD_ERR_ARG outside those ranges. */
int afd_set_walk_limits(afd_ctx *ctx, int64_t iter_cap, int32_t stack_cap,
                        int64_t arena_chunks_max);

/* Wait for the context's stream and return the device status word. */
int afd_sync(afd_ctx *ctx);

/* Sizes of the current tree and lists: out[0] n, [1] cells, [2] groups,
 * [3] EPJ entries, [4] SPJ entries, [5] interactions of one force
 * evaluation (sum over groups of n_i * (n_epj + n_spj)), [6] lists saved
 * for reuse (0/1), [7] deepest level, [8] kernels launched by this context
 * so far, [9] force-kernel work units (32-particle group chunks). Host
 * array of 10 int64. */
int afd_stats(afd_ctx *ctx, int64_t *out);

/* Copy an internal array to host memory for inspection and parity tests.
 * With host_buf NULL only *bytes is set to the size needed. Synchronises.
 * Items and element types:
 *   ROOT        systems x 4 x f64 (centre x, y, z, side L)
 *   KEYS        n x u64 sorted Morton keys
 *   PERM        n x u32 caller index of each Morton position
 *   CELL_LEVEL  cells x u32      CELL_FIRST  cells x u32
 *   CELL_COUNT  cells x u32      CELL_SKIP   cells x u32 (pre-order end of subtree)
 *   CELL_PARENT cells x u32 (0xffffffff for the root)
 *   CELL_CHILD  cells x 8 x u32 (by octant, 0xffffffff when empty)
 *   CELL_MASS   cells x f64      CELL_COM    cells x 3 x f64
 *   CELL_QUAD   cells x 6 x f64 (xx yy zz xy xz yz; zeros when monopole)
 *   GROUP_FIRST groups x u32     GROUP_COUNT groups x u32
 *   GROUP_BOX   groups x 6 x f64 (min x y z, max x y z)
 *   GROUP_SELF  groups x u32: 1 + position of the group's first particle in
 *               its EPJ list (its particles follow contiguously; the force
 *               kernel skips each particle's own pair there), 0 if absent
 *   EPJ_OFF / SPJ_OFF (groups + 1) x u64, EPJ_IDX / SPJ_IDX entries x u32
 *   NBR_OFF (groups + 1) x u64, NBR_IDX entries x u32 (neighbour lists)
 *   CELL_TBOX   cells x 8 x f32 (tight box: min x y z, 0, max x y z, 0)
 *   GROUP_SBOX  groups x 6 x f32 (search box: min x y z, max x y z)
 * Cells are numbered in depth-first pre-order, children in Morton order. */
typedef enum {
  AFD_EXPORT_ROOT = 0,
  AFD_EXPORT_KEYS = 1,
  AFD_EXPORT_PERM = 2,
  AFD_EXPORT_CELL_LEVEL = 3,
  AFD_EXPORT_CELL_FIRST = 4,
  AFD_EXPORT_CELL_COUNT = 5,
  AFD_EXPORT_CELL_SKIP = 6,
  AFD_EXPORT_CELL_PARENT = 7,
  AFD_EXPORT_CELL_CHILD = 8,
  AFD_EXPORT_CELL_MASS = 9,
  AFD_EXPORT_CELL_COM = 10,
  AFD_EXPORT_CELL_QUAD = 11,
  AFD_EXPORT_GROUP_FIRST = 12,
  AFD_EXPORT_GROUP_COUNT = 13,
  AFD_EXPORT_GROUP_BOX = 14,
  AFD_EXPORT_GROUP_SELF = 15,
  AFD_EXPORT_EPJ_OFF = 16,
  AFD_EXPORT_EPJ_IDX = 17,
  AFD_EXPORT_SPJ_OFF = 18,
  AFD_EXPORT_SPJ_IDX = 19,
  AFD_EXPORT_NBR_OFF = 20,
  AFD_EXPORT_NBR_IDX = 21,
  AFD_EXPORT_CELL_TBOX = 22,
  AFD_EXPORT_GROUP_SBOX = 23
} afd_export_item;

int afd_export(afd_ctx *ctx, int what, void *host_buf, size_t *bytes);

/* Milliseconds of the most recent force kernel launch as measured by CUDA
 * events recorded around it on the context's stream (synchronises). */
int afd_last_force_ms(afd_ctx *ctx, float *ms);

/* Root cell of a particle set without any device allocation.
 *
 * The paper has no counterpart: this entry point is for callers that cannot
 * allocate device memory -- code whose GPU memory is entirely owned by
 * another allocator (for example a framework's memory pool), or loops that
 * must not call cudaMalloc / cudaFree after start-up because those calls can
 * synchronise the device. It needs no context (afd_create allocates).
 *
 * Computes the same root cell as afd_tree_build, bit for bit (the same
 * reduction on order-preserving integer keys of the doubles, so a zero
 * centre has the same sign) -- centre (min + max) / 2 per axis, side = the
 * smallest power of two >= 1.000001 x the largest extent (1 for a zero
 * extent; root (0, 0, 0, 1) for n = 0) -- from x, y, z (n device doubles
 * each, caller order), and checks m (n device doubles) for finiteness.
 * root_out: device, 4 doubles (centre x, y, z, side). nonfinite_out: device
 * int, set to 1 when a coordinate or mass is NaN or infinite (NaN
 * coordinates are then left out of the box) or when no finite power of two
 * reaches 1.000001 x the extent (finite coordinates such as +-1e308; the
 * side is then +inf), else 0. Queued on `stream` (a cudaStream_t; NULL = the
 * legacy default stream); the call does not synchronise.
 *
 * Scratch: a file-scope static device array of 29,440 bytes, which every GPU
 * that loads the library keeps until the process exits. All calls on a
 * device share it and it keeps the last call's contents; each call clears
 * the part that must start at zero. Calls whose work overlaps on the GPU
 * (different streams or host threads) race on it: serialise them. The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; the lookup is not
 * stream-ordered, so make that first call before any stream capture. The
 * address is kept for the life of the process: do not use this entry point
 * on a device after cudaDeviceReset in the same process.
 *
 * n must lie in 0 .. 2^31 - 1 (the library's particle index range); a larger
 * n returns AFD_ERR_TOO_LARGE before the device is touched. The call makes no
 * cudaMalloc, cudaFree or other allocating call. */
int afd_root_cell_static(const double *x, const double *y, const double *z, const double *m,
                         int64_t n, double *root_out, int *nonfinite_out, void *stream);

/* Measured FP32 rate of device `device` in TFLOP/s: the F_GPU of the force
 * kernel model (Appendix A, Eq. model_kernel), from a kernel of independent
 * packed FP32 FMA chains timed with CUDA events on `stream` (best of three
 * launches; synchronises; allocates 4 bytes of scratch). Reported next to the
 * nominal peak (SMs x 128 lanes x 2 flops x clock) in benchmarks. */
int afd_fp32_peak(int device, void *stream, double *tflops_out);

/* ---------------------------------------------------------------------------
 * Learned opening criterion.
 *
 * Not in the paper, which accepts a cell by its opening angle alone (the
 * "standard Barnes-Hut scheme", Section 2; theta, Section 6.1). A small
 * network scores a (group, cell) pair from size, distance and multipole
 * moments and predicts the log2 of the largest relative force error, over
 * the group's particles, that replacing the cell's particles by its
 * superparticle would cause. The walk (afd_make_interaction_lists) then
 * decides a cell c for group g as follows, in FP32:
 *   - open c if it holds g's first particle;
 *   - accept c if s^2 < theta_lo^2 d^2 (s cell side, d COM-to-box distance);
 *   - open c unless s^2 < theta_hi^2 d^2;
 *   - otherwise accept c iff the network's output < tau.
 * Features (8, FP32): log2(s/d), log2(M / (d^2 A_g)), log2(|Q|_F / (M s^2)),
 * log2(e/d), log2(n_c), log2(eps/d), u.Q.u / (|u|^2 |Q|_F), log2(|u|/d),
 * each clamped to [-32, 32] -- M, Q, n_c the cell's mass, traceless
 * quadrupole and particle count, A_g the smallest reference |a| among the
 * group's particles, e half the group box diagonal, u = box centre - COM.
 * log2 is a fixed polynomial (exponent + t p(t) on the mantissa 1 + t).
 * Network: 8-32-32-1, ReLU, FP16 parameters; inputs RN16((f - mu) * isd)
 * and first-layer activations RN16(min(max(., 0), 65504)) in FP16 (RN16:
 * nearest FP16, ties to even), sums in FP32 (products of FP16 values are
 * exact); the walk evaluates it on the tensor cores, sixteen pairs per
 * warp instruction sequence, summing in the tensor core's order. Training
 * (afd_mlp_loss_grad, afd_mlp_train) uses the same network with FP32 inputs
 * and activations. Without weights (afd_mac_set) or reference magnitudes
 * for the current particles, the walk uses theta.
 *
 * Parameter vector (AFD_MAC_PARAMS floats): mu[8] isd[8] W1[32][8] b1[32]
 * W2[32][32] b2[32] w3[32] b3[1], row-major (W[j][k]: unit j, input k).
 * ------------------------------------------------------------------------- */
#define AFD_MAC_FEATURES 8
#define AFD_MAC_HIDDEN 32
#define AFD_MAC_PARAMS 1393

/* Install the network (params: host, AFD_MAC_PARAMS floats, rounded to FP16
 * on the device) and the band [theta_lo, theta_hi] and threshold tau; params
 * NULL removes it (theta criterion). The context must have been created
 * with cfg.mac = 1. Synchronises. */
int afd_mac_set(afd_ctx *ctx, const float *params, double theta_lo, double theta_hi, double tau);

/* Reference acceleration magnitudes for feature 2 and the targets: amag,
 * device, n floats, caller order (copied). With cfg.mac = 1 every force
 * evaluation also stores |a| of its result here, so later construction
 * steps use the latest accelerations. Does not synchronise. */
int afd_mac_set_reference(afd_ctx *ctx, const float *amag, int64_t n);

/* Training samples from the current tree (needs cfg.mac = 1, a tree and
 * reference magnitudes for its particles, else AFD_ERR_NO_TREE /
 * AFD_ERR_NO_REFERENCE). The pairs are those the criterion would leave to the
 * network: a walk per group that accepts below theta_lo and opens every
 * other cell records each visited cell in [theta_lo, theta_hi). A pair is
 * kept when keep >= 1, or when a fixed hash of (seed, group, cell) falls
 * below keep * 2^32. For the first min(total, cap) kept pairs, in group
 * order: feat (device, cap x 8 floats) gets the features and label (device,
 * cap floats) the target -- log2 of max over the group's particles of
 * |a_cell - a_exact| / |a_ref| (superparticle term, with the quadrupole when
 * cfg.multipole = 1, against the direct sum over the cell's particles),
 * clamped to [-40, 8]. pair (device, cap x 2 u32 (group, cell), or NULL)
 * receives the pairs. *n_out (host) = total kept pairs, which may exceed
 * cap. Synchronises. */
int afd_mac_samples(afd_ctx *ctx, double theta_lo, double theta_hi, double keep, uint64_t seed,
                    int64_t cap, float *feat, float *label, uint32_t *pair, int64_t *n_out);

/* out (host, 5 int64): [0] the last walk used the learned criterion (0/1),
 * [1] network evaluations in it, [2] cells the network accepted, [3]
 * reference magnitudes present for the current particles (0/1), [4] warp
 * steps of the walk that evaluated the network (so [1] / [4] is the mean
 * number of lanes busy per evaluation round). Synchronises when [0] is 1. */
int afd_mac_info(afd_ctx *ctx, int64_t *out);

/* The network's output for n feature rows (feat: device, n x 8 floats; out:
 * device, n floats), with params (host) rounded to FP16, computed by the
 * walk's own tensor-core code (the same outputs bit for bit). Queued on
 * `stream` (a cudaStream_t, NULL = legacy default); synchronises it. */
int afd_mlp_forward(const float *params, const float *feat, int64_t n, float *out, void *stream);

/* Mean squared error of the network (FP32 parameters, not rounded) on n
 * device samples, and its gradient with respect to every parameter (host,
 * AFD_MAC_PARAMS floats; zero for mu and isd, which are not trained). The
 * forward and backward passes are this library's kernels; the block partial
 * sums are reduced in a fixed order. 1 <= n <= 2^24. Synchronises. */
int afd_mlp_loss_grad(const float *params, const float *feat, const float *label, int64_t n,
                      float *grad, float *loss, void *stream);

/* Train the network on n device samples (feat n x 8, label n): mu and isd
 * from the feature statistics (FP16 values), b3 from the mean target,
 * He-normal weights from `seed`; then `epochs` passes of Adam (lr with a
 * cosine decay to 5%, betas 0.9 / 0.999) over minibatches of `batch`
 * (1 .. 65536) in a fresh seeded order per epoch, minimising the mean
 * squared error. params (host, AFD_MAC_PARAMS floats) receives the FP32
 * result; loss_hist (host, epochs floats, may be NULL) each epoch's mean
 * minibatch loss. Deterministic for a given seed. Synchronises. */
int afd_mlp_train(const float *feat, const float *label, int64_t n, int epochs, int batch,
                  double lr, uint64_t seed, float *params, float *loss_hist, void *stream);

/* FP64 direct summation (G = 1, Plummer softening eps, j != i, pairs at zero
 * softened distance skipped) for n_t targets: out (device, n_t x 4 doubles)
 * = (ax, ay, az, phi) of particle targets[t] (device u32 indices < n; a
 * target >= n gives NaN) from the n particles x, y, z, m (device). Queued on
 * `stream`; does not synchronise. */
int afd_direct_sum(const double *x, const double *y, const double *z, const double *m, int64_t n,
                   const uint32_t *targets, int64_t n_t, double eps, double *out, void *stream);

/* Measured rates of the instruction streams the kernels use, each from
 * independent chains timed with CUDA events on `stream` (best of three
 * launches; synchronises; allocates 4 bytes): out (host, 4 doubles) = [0]
 * packed fma.rn.f32x2 TFLOP/s, [1] scalar FP32 FMA TFLOP/s, [2] MUFU
 * rsqrt.approx.f32 lane-operations per second / 1e12, [3] packed
 * fma.rn.f16x2 TFLOP/s (2 flops per lane-FMA). */
int afd_pipe_rates(int device, void *stream, double *out);

/* Human-readable text for a status code (static storage). */
const char *afd_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* AFDPS_H */
