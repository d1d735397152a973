/*
 * greem.h -- C ABI of the GB300-native periodic short-range tree force of GreeM
 * (Ishiyama, Fukushige & Makino 2009, "GreeM: Massively Parallel TreePM Code for
 * Large Cosmological N-body Simulations").
 *
 * What the library computes (paper passages in brackets):
 *   acc_i = sum_j m_j g_P3M(|d_ij|/eta) d_ij / |d_ij|^3          [Sec. 2.1, Eq. 1]
 *   g_P3M = the S2 cutoff of Hockney & Eastwood, zero for R >= 2  [Sec. 2.1, Eq. 2]
 *   eta = r_cut / 2                                               [Sec. 2.2, step 1]
 * evaluated with a tree (Barnes-Hut opening angle theta, nodes farther than r_cut
 * pruned) over Barnes' grouped interaction lists (groups of at most n_crit
 * particles share one list) with periodic images                [Sec. 2.2, steps 2-5;
 * Sec. 3.1.2; Sec. 1 on image particles].  The pairwise arithmetic runs in FP32 on
 * coordinates relative to each group's centre                   [Sec. 3.1.1].
 * G = 1.  Masses, positions and L are in any consistent units.
 *
 * Conventions for every call:
 *  - pos is [N,3] float64 row-major, mass is [N] float32, acc is [N,3] (float32, or
 *    float64 for GREEM_F64), all CONTIGUOUS DEVICE pointers owned by the caller (HOST
 *    pointers in greem_short_force_host only).  The library never frees them and does
 *    not keep them after the call returns, except the pointers captured by
 *    greem_graph_capture (see there).
 *  - acc is written in INPUT order.  Positions outside [0, L) are wrapped (periodic);
 *    they are not errors.
 *  - Work is enqueued on the context's stream.  Calls that return a status wait for
 *    the stream, because capacity and input errors are detected on the device.
 *  - A context is not thread-safe; use one per host thread.
 *  - No C++ exception crosses this interface.  Every call returns GREEM_OK (0) or a
 *    negative GREEM_ERR_* code; greem_strerror() describes it.
 */
#ifndef GREEM_H
#define GREEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define GREEM_OK 0
#define GREEM_ERR_INVALID_ARG -1   /* bad size/parameter, or a NaN/Inf position or a mass that is
                                      NaN or of magnitude >= 2^38 seen on the device */
#define GREEM_ERR_CUDA -2          /* a CUDA runtime call failed */
#define GREEM_ERR_OOM -3           /* device or host allocation failed */
#define GREEM_ERR_CAPACITY -4      /* a device buffer overflowed: from graph replays, or from a
                                      direct call still overflowing after its retries (direct
                                      calls grow their buffers and retry, 6 attempts in all) */
#define GREEM_ERR_TIMEOUT -5       /* a bounded device wait gave up; the context stays usable */
#define GREEM_ERR_NOT_IMPLEMENTED -6

/* Force precision (greem_params.precision). */
#define GREEM_F32_REL 0  /* FP32 pairwise arithmetic on group-relative coordinates (default) */
#define GREEM_F64 1      /* plain FP64 form on the same lists; acc is float64 [N,3] */

/* greem_params.flags */
#define GREEM_FLAG_INDEX_LISTS 1u  /* also keep the interaction lists as (kind, index, image)
                                      entries so that greem_debug_dump(GREEM_DUMP_LISTS) works */
#define GREEM_FLAG_STAGE_TIMES 2u  /* record per-stage device times in greem_stats */
#define GREEM_FLAG_ADD_PM 4u       /* add the PM (long-range) force of greem_pm_force, on n_pm^3 with
                                      the assign scheme, to acc in the same call (single box, FP32):
                                      the full TreePM force, Sec. 2.1 */
#define GREEM_FLAG_QUADRUPOLE 16u  /* add the second-order (quadrupole) terms of accepted nodes,
                                      with the derivatives of the cutoff function (Sec. 4.1):
                                      1/2 B tr(Q) d + 1/2 C (d.Q.d) d + B Q d, B = A'/r, C = B'/r,
                                      A = g(r/eta)/r^3, Q the node's second moments about its COM
                                      (FP32).  FP32 precision and eps = 0 only (INVALID_ARG
                                      otherwise); keeps the index lists as INDEX_LISTS does. */
#define GREEM_FLAG_THETA_EQ12 8u   /* distance-dependent opening angle of Sec. 4.1, Eq. 12: a node is
                                      accepted iff l < theta(d) d with theta(d) = min(theta,
                                      theta0 / sqrt(R g(R))), R = d/eta, g of Eq. 2 (theta(d) = theta
                                      where R g(R) = 0); theta is then the upper limit the paper
                                      calls for.  Per box in greem_short_force_batched (theta0 from
                                      each box's parameters, the flag from per_box[0]). */

/* PM mass assignment schemes (greem_pm_force, greem_params.assign). */
#define GREEM_ASSIGN_CIC 0
#define GREEM_ASSIGN_TSC 1         /* the paper's choice (Sec. 2.2 step 1) */

typedef struct greem_params {
    double L;        /* periodic box side, > 0 */
    double r_cut;    /* cutoff radius, 0 < r_cut < L/2; eta = r_cut/2 (Sec. 2.2 step 1) */
    double theta;    /* opening angle, >= 0 (theta = 0 opens every node within r_cut) */
    double eps;      /* Plummer softening, >= 0; 0 gives Eq. 1 exactly.  With eps > 0 the
                        pair term is m g(r/eta) d / (r^2+eps^2)^(3/2). */
    int n_crit;      /* group size bound N_crit (Sec. 3.1.2), >= 1 */
    int n_leaf;      /* leaf bound N_leaf: a node is a leaf when it holds fewer (Sec. 3.1.2), >= 1 */
    int precision;   /* GREEM_F32_REL or GREEM_F64 */
    int list_chunk;  /* list entries staged per force-kernel chunk: 0 = default (256); power of
                        two in [64, 2048] */
    int block_shape; /* warps per force-kernel block: 0 = default (16); 1..16; block_shape x
                        list_chunk x 32 bytes (two chunk buffers per warp) must not exceed
                        226 KB of shared memory */
    unsigned flags;  /* GREEM_FLAG_* */
    int n_pm;        /* PM grid points per side for GREEM_FLAG_ADD_PM (8..1024) */
    int assign;      /* GREEM_ASSIGN_CIC or GREEM_ASSIGN_TSC for GREEM_FLAG_ADD_PM */
    double theta0;   /* theta_0 of Eq. 12 for GREEM_FLAG_THETA_EQ12, > 0 (R in units of eta
                        makes it dimensionless) */
} greem_params;

/* Fills defaults: L 1, r_cut 3/32, theta 0.5, eps 0, n_crit 64, n_leaf 10 (Sec. 3.1.2),
 * F32 precision, default chunk and block shape, no flags, theta0 0.25. */
void greem_params_default(greem_params *p);

typedef struct greem_ctx greem_ctx; /* opaque; owns all device workspace */

/* Creates a context on the CURRENT CUDA device that enqueues on cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream).  Errors: GREEM_ERR_INVALID_ARG when
 * out is NULL, GREEM_ERR_CUDA when no device is usable, GREEM_ERR_OOM. */
int greem_create(greem_ctx **out, void *cuda_stream);

/* Frees the context and all of its device memory (after waiting for its stream). */
void greem_destroy(greem_ctx *ctx);

/* Steps S1-S4 for one box: wrap and 63-bit Morton keys (Sec. 3.2.5), stable radix sort,
 * octree with N_leaf leaves and FP64 monopole moments (Sec. 2.2 step 2; Sec. 3.1.2), and
 * the groups of at most n_crit particles (Sec. 2.2 step 5).  The tree lives in the
 * context until the next build or force call and can be read with greem_debug_dump.
 * Errors: INVALID_ARG (N < 1, N >= 2^31, L <= 0, r_cut outside (0, L/2), theta < 0,
 * eps < 0, n_crit < 1, n_leaf < 1, a NaN/Inf position, a mass that is NaN or of
 * magnitude >= 2^38: the FP32 force keeps the zero-distance pair of a particle with
 * itself finite only below that), CUDA, OOM. */
int greem_build_tree(greem_ctx *ctx, const double *pos, const float *mass, int64_t N, const greem_params *p);

/* The whole short-range force (S1-S6) with default settings: n_leaf 10, eps 0, FP32
 * relative-coordinate arithmetic.  Uses a context owned by the library for the current
 * device, on the legacy default stream.  acc: float32 [N,3] device, input order.
 * Errors as greem_build_tree. */
int greem_short_force(const double *pos, const float *mass, int64_t N, double L, double r_cut, double theta,
                      int n_crit, float *acc);

/* The whole short-range force with explicit parameters.  acc is float32 [N,3] for
 * GREEM_F32_REL and float64 [N,3] for GREEM_F64.  Errors as greem_build_tree.
 * A call that repeats one of the two previous calls on this context (the same pos, mass
 * and acc pointers, N and parameters; new contents of pos and mass are fine) runs as one CUDA
 * graph launch of the whole step from the third such call on: the same kernels and
 * results, without the per-kernel launch cost.  If the new positions need more buffer
 * space than the graph was captured with, the call falls back to the usual path, which
 * grows the buffers and retries.  Calls with GREEM_FLAG_ADD_PM never replay;
 * greem_debug_set(GREEM_DEBUG_REPLAY, 0) turns replays off.  greem_stats.replayed tells
 * whether the last call replayed (stage times are measured in replays too). */
int greem_short_force_ex(greem_ctx *ctx, const double *pos, const float *mass, int64_t N, const greem_params *p,
                         void *acc);

/* nstep independent short-range force problems whose inputs and results live in HOST
 * memory, each one greem_short_force_ex with the same p.  Problem k reads pos[k]
 * (float64 [N[k],3]) and mass[k] (float32 [N[k]]) and writes acc[k] (float32 or
 * float64 [N[k],3] by p->precision), all host pointers owned by the caller.  The copies
 * overlap the computation: while problem k runs on the context's stream, the inputs of
 * k+1 are copied in and the result of k-1 is copied out on two more streams, through
 * two device staging slots that the context keeps (about 40 bytes per particle each,
 * sized for the largest N seen).  The overlap needs page-locked host memory
 * (cudaHostAlloc, cudaHostRegister, or torch pin_memory); pageable pointers work but
 * their copies do not overlap.  Returns when every result is in host memory, or at the
 * first failing problem: its code is returned, its acc and those of later problems are
 * not written, and earlier ones are complete.  The statistics are those of the last
 * problem run.  Errors as greem_short_force_ex, plus INVALID_ARG for nstep < 1 or a NULL
 * array or pointer. */
int greem_short_force_host(greem_ctx *ctx, int nstep, const double *const *pos, const float *const *mass,
                           const int64_t *N, const greem_params *p, void *const *acc);

/* nbox independent periodic boxes in one pass: box b holds particles
 * [offsets[b], offsets[b+1]) of pos/mass/acc and uses per_box[b] (every box may have
 * its own L, r_cut, theta, eps, n_crit, n_leaf; precision, list_chunk, block_shape and
 * flags are taken from per_box[0]).  offsets is a HOST array of nbox+1 increasing
 * values with offsets[0] = 0.  One sort, one tree pass, one list pass and one
 * persistent force launch serve all boxes.  Errors as greem_build_tree, plus
 * INVALID_ARG for nbox < 1, nbox > 65536 or an empty box. */
int greem_short_force_batched(greem_ctx *ctx, int nbox, const int64_t *offsets, const double *pos,
                              const float *mass, const greem_params *per_box, void *acc);

/* PM (long-range) part of the TreePM split (Sec. 2.1; Sec. 2.2 step 1; Table 2): mass
 * assigned to an n_pm^3 periodic grid (points at j L/n_pm) with CIC or TSC, FFT (cuFFT,
 * FP32), convolution with G(k) = -4 pi S(k eta)^2 / (k^2 W(k)^2) where S is the transform
 * of the S2 cloud of radius eta = r_cut/2 (so that PP of Eq. 1-2 plus PM is Newton's law)
 * and W the assignment window (deconvolved twice), k = 0 removed, spectral gradient,
 * interpolation with the same weights.  pos/mass/acc_pm as for the short-range calls
 * (device, input order); acc_pm is float32 [N,3] and is overwritten.  Errors:
 * INVALID_ARG (N < 1, L <= 0, n_pm outside 8..1024, r_cut outside (0, L/2), unknown
 * assign), CUDA, OOM. */
int greem_pm_force(greem_ctx *ctx, const double *pos, const float *mass, int64_t N, double L, int n_pm,
                   double r_cut, int assign, float *acc_pm);

/* Captures the whole short-range force for (pos, mass, N, p, acc) into a CUDA graph held by
 * the context.  Runs the call once first (sizing every buffer), then records it.  The graph
 * keeps the device pointers pos, mass and acc: they must stay valid, and their CONTENTS are
 * read at each greem_graph_launch.  Errors as greem_short_force_ex. */
int greem_graph_capture(greem_ctx *ctx, const double *pos, const float *mass, int64_t N, const greem_params *p,
                        void *acc);

/* Replays the captured graph and waits for it.  Returns GREEM_ERR_CAPACITY when the new
 * positions need more tree, group or list space than was captured (capture again), and
 * GREEM_ERR_INVALID_ARG when no graph was captured or a NaN/Inf position was seen. */
int greem_graph_launch(greem_ctx *ctx);

typedef struct greem_stats {
    int64_t n_particles;
    int64_t n_boxes;
    int64_t n_nodes;          /* tree nodes over all boxes */
    int64_t n_groups;         /* interaction-list groups */
    int64_t n_list_entries;   /* sum over groups of the list length (unpadded) */
    int64_t n_interactions;   /* sum over groups of n_g x list length (unpadded): the N_int sum */
    int64_t n_evaluated;      /* pair evaluations the force kernel performed (padded lists) */
    int64_t list_capacity;    /* entries in the list pool */
    int64_t kernel_launches;  /* kernels launched by the last call */
    int32_t l_min;            /* shallowest group level of box 0 */
    int32_t retries;          /* capacity retries of the last call */
    /* with STAGE_TIMES, by events on the context's stream: keys; sort and gather; tree,
     * moments and node COM offsets; groups (particle offsets and groups run on a second
     * stream beside the moments: what remains of them after the moments, and the
     * second-order moments); lists; force (and PM); total */
    double ms_keys, ms_sort, ms_tree, ms_groups, ms_lists, ms_force, ms_total;
    /* list walks that started below the root, from the level-K cell table (Sec. 3.1.2
     * walk; the conditions under which the entries are the same are in lists.cu), and the
     * leaves above level K those walks took from the table (counted only by calls that
     * build index lists, GREEM_FLAG_INDEX_LISTS, 0 otherwise; a group whose list is
     * walked again into fresh pages counts its leaves twice) */
    int64_t n_start_table, n_start_coarse;
    int64_t replayed;  /* 1 if the last greem_short_force_ex call replayed its graph, else 0 */
} greem_stats;

/* Counters of the last call.  Errors: INVALID_ARG for NULL arguments. */
int greem_get_stats(greem_ctx *ctx, greem_stats *out);

/* Debug dumps of the last build/force call into host memory. */
#define GREEM_DUMP_KEYS 0      /* uint64 [N] sorted Morton keys */
#define GREEM_DUMP_PERM 1      /* uint32 [N] sorted position -> input index */
#define GREEM_DUMP_NODES 2     /* int64 [n_nodes, 9]: level, ix, iy, iz (cell index at its level),
                                  begin, end, skip, leaf, parent (-1 for a root); preorder */
#define GREEM_DUMP_MOMENTS 3   /* float64 [n_nodes, 4]: M, cx, cy, cz */
#define GREEM_DUMP_GROUPS 4    /* int64 [n_groups]: node index of each group, preorder */
#define GREEM_DUMP_LIST_OFFSETS 5 /* int64 [n_groups+1]: CSR offsets into GREEM_DUMP_LISTS */
#define GREEM_DUMP_LISTS 6     /* int64 [n_entries, 5]: kind (0 particle, 1 node), index (sorted
                                  particle or node), image shift x, y, z in units of L (needs
                                  GREEM_FLAG_INDEX_LISTS on the force call) */
#define GREEM_DUMP_QUADRUPOLES 7 /* float64 [n_nodes, 6]: second moments xx, yy, zz, xy, xz, yz about
                                    the COM (after a call with GREEM_FLAG_QUADRUPOLE) */
/* Copies the array into host_buf when cap_bytes suffices; *len_bytes always gets the size.
 * Errors: INVALID_ARG (unknown what, no previous call, cap too small -> *len_bytes set). */
int greem_debug_dump(greem_ctx *ctx, int what, void *host_buf, int64_t cap_bytes, int64_t *len_bytes);

/* The interaction lists of selected groups only (for sampled checks at sizes where the
 * whole list dump would not fit in host memory).  groups: HOST int64 [ngroups] group
 * indices (0 <= g < n_groups of the last force call, which must have used
 * GREEM_FLAG_INDEX_LISTS).  offsets: HOST int64 [ngroups+1] CSR offsets (written);
 * entries: HOST int64 [cap_entries, 5] as GREEM_DUMP_LISTS, each list in preorder.
 * *n_entries always gets the total.  Errors: INVALID_ARG (no lists, bad group index,
 * cap_entries too small), CUDA. */
int greem_debug_dump_group_lists(greem_ctx *ctx, const int64_t *groups, int64_t ngroups, int64_t *offsets,
                                 int64_t *entries, int64_t cap_entries, int64_t *n_entries);

/* Failure-path controls, for tests of the error handling described above.  The paper
 * has no counterpart: they exist so that every recovery path (capacity growth and
 * retry, the retry bound, a bounded device wait that gives up) can be exercised without
 * a GPU fault.  Each applies to this context only:
 *   GREEM_DEBUG_WAIT_POLLS    the polls each list-chunk wait of the FP32 force kernel makes
 *                             before it gives up (default 2^22): with 0 every call that
 *                             streams a list returns GREEM_ERR_TIMEOUT, after the warp has
 *                             let its copies land, and the context stays usable; value < 0
 *                             restores the default.  Stays in effect until changed.
 *   GREEM_DEBUG_NODE_CAP      starting tree-node capacity of the NEXT call (> 0)
 *   GREEM_DEBUG_LIST_CAP      starting list-pool capacity, in entries, of the NEXT call (> 0)
 *   GREEM_DEBUG_STACK_CAP     starting traversal-stack entries per list warp, from the NEXT
 *                             call on (> 0)
 *                             (a call that overflows a capacity grows it and retries, as it
 *                             does from the usual first guesses; greem_stats.retries counts)
 *   GREEM_DEBUG_MAX_ATTEMPTS  attempts per call before GREEM_ERR_CAPACITY is returned
 *                             (default 6; value < 1 restores it).  Stays in effect.
 *   GREEM_DEBUG_REPLAY        1 (default): repeated greem_short_force_ex calls replay a
 *                             graph of the call; 0: they do not.  Stays in effect.
 *   GREEM_DEBUG_START_LEVEL   the deepest level (<= 7) at which a list walk may start
 *                             instead of the root (default 7; 0 or 1: every walk starts at
 *                             the root; value < 0 restores the default).  The lists hold the
 *                             same entries either way; for timing comparisons.  Stays in effect.
 * Every setting also drops the graph that repeated greem_short_force_ex calls replay.
 * Errors: INVALID_ARG (NULL ctx, unknown what, value out of range). */
#define GREEM_DEBUG_WAIT_POLLS 0
#define GREEM_DEBUG_NODE_CAP 1
#define GREEM_DEBUG_LIST_CAP 2
#define GREEM_DEBUG_STACK_CAP 3
#define GREEM_DEBUG_MAX_ATTEMPTS 4
#define GREEM_DEBUG_START_LEVEL 5
#define GREEM_DEBUG_REPLAY 6
int greem_debug_set(greem_ctx *ctx, int what, int64_t value);

/* The FP32 list entries of selected groups exactly as the force kernel reads them, for
 * entry-level checks of the list builder as the FP32 force runs it (Sec. 3.1.1: positions
 * relative to the group's centre; Sec. 2.2 step 5: one list per group).  Works after any
 * force call.  Per group the unpadded list in the builder's own order (not sorted):
 * entries is HOST float32 [cap_entries, 4], each (x, y, z) = the entry's position (a
 * particle, or a node's centre of mass, shifted by its periodic image) minus the centre of
 * the group's cell, in units of r_cut, and w = the mass.  index_entries, when not NULL,
 * gets the matching HOST int64 [cap_entries, 5] entries (as GREEM_DUMP_LISTS) in the same
 * order; it needs a last call with GREEM_FLAG_INDEX_LISTS.  groups, offsets and
 * *n_entries as greem_debug_dump_group_lists.  Errors: INVALID_ARG (no lists, index
 * entries asked for without index lists, bad group index, cap_entries too small), CUDA. */
int greem_debug_dump_group_entries(greem_ctx *ctx, const int64_t *groups, int64_t ngroups, int64_t *offsets,
                                   float *entries, int64_t *index_entries, int64_t cap_entries,
                                   int64_t *n_entries);

/* Picks n_crit from candidates[0..ncand) (ncand = 0 -> 32, 48, 64, 96, 128, 160, 192, 256,
 * 384, 512) at p's list_chunk and block_shape, then list_chunk and block_shape at that n_crit,
 * then re-times the neighbouring n_crit candidates at the chosen shape; each setting is
 * timed on the whole force over these inputs (best of three calls).  Writes the best
 * parameters to *best (a copy of *p with those three fields set).  acc is scratch output
 * of the right type.  Errors as greem_short_force_ex. */
int greem_autotune(greem_ctx *ctx, const double *pos, const float *mass, int64_t N, const greem_params *p,
                   const int *candidates, int ncand, void *acc, greem_params *best);

/* The pairwise FP32 kernel on its own, for the pairwise-error experiment of Sec. 3.1.1:
 * for every pair k, the force on x_i[k] from a particle of mass m_j[k] at x_j[k] with
 * both positions passed relative to the group centre x_g[k] (no periodic wrap).  All
 * arrays are device: x_g, x_i, x_j float64 [npairs,3], m_j float32 [npairs], acc float32
 * [npairs,3].  Errors: INVALID_ARG (npairs < 1, r_cut <= 0, eps < 0). */
int greem_pair_force_f32(greem_ctx *ctx, const double *x_g, const double *x_i, const double *x_j, const float *m_j,
                         int64_t npairs, double r_cut, double eps, float *acc);

/* The pairwise FP32 force of greem_pair_force_f32 for callers that cannot allocate
 * device memory (a library whose allocator policy forbids driver allocations, work that
 * must not be held up by the device-wide synchronisation cudaMalloc/cudaFree can
 * impose, a process whose free memory belongs to another allocator).  The paper has no
 * counterpart: it is a deployment variant.  It allocates nothing: its scratch is a
 * file-scope device array sized for at most 32768 pairs (about 6.5 MB, held on every GPU
 * that loads the library until exit).  The caller passes inputs and output as for
 * greem_pair_force_f32, plus the stream to run on (NULL = legacy default stream).  Every
 * call waits for that stream, and only that stream, to read its status word.  The first
 * call on each device looks up the array's device address and should come before any
 * stream capture.  All calls on a device share the array (it keeps the last call's
 * contents); calls that overlap on the GPU race, so serialise them.
 * Errors: INVALID_ARG (npairs < 1 or > 32768, r_cut <= 0, eps < 0, NULL pointer), CUDA,
 * TIMEOUT. */
int greem_pair_force_f32_noalloc(const double *x_g, const double *x_i, const double *x_j, const float *m_j,
                                 int64_t npairs, double r_cut, double eps, float *acc, void *cuda_stream);

/* ---- Several processes on one box (Sec. 2.2 steps 3, 4 and 7; Sec. 2.3.1) -----------------
 * The paper divides the periodic box into p subboxes by recursive multisection, one per
 * process, with boundaries set by sampled particles (Sec. 2.3.1).  Each process builds the
 * tree of its own particles, sends every other process the local essential tree (LET) that
 * process needs, and computes the force on its particles from a tree of its particles and
 * the items it received (steps 3-5).  The calls below are the per-process pieces; the data
 * exchange between processes is the caller's (an all-to-all of the counts and items).
 *
 * A domain box is int32 [6] = (xlo, xhi, ylo, yhi, zlo, zhi) in finest cells (L/2^21, the
 * cells of the Morton key), half-open per axis, 0 <= lo <= hi <= 2^21; a particle belongs
 * to the box that holds its finest cell.  A set of boxes (at most 1024) must tile the
 * periodic box. */

/* Eq. 3-5: the number of particles a process samples for the next decomposition.
 * n_samp = N R f with f = t_local / t_sum (Eq. 4, the process's share of the measured
 * force time; f = 1/nproc when t_sum <= 0, before any time is measured), raised to
 * n_local R / (1 + alpha) when that is larger (Eq. 5; alpha < 0 leaves the lower limit
 * out), rounded, and capped at n_local.  Host only.  Returns the count, or -1 for invalid
 * arguments (n_total < 0, n_local outside [0, n_total], nproc < 1, rate < 0 or not finite). */
int64_t greem_sample_count(int64_t n_total, int64_t n_local, int nproc, double rate, double t_local, double t_sum,
                           double alpha);

/* Recursive multisection of the sampled particles (Sec. 2.2; Sec. 2.3.1): cells (HOST int32
 * [n, 3], the samples' finest cells, from greem_cell_index on every process, gathered) are
 * cut along x into px slabs holding equal numbers of samples, each slab along y into py
 * columns, each column along z into pz boxes.  A cut lies between the two samples that the
 * equal split separates (rounded up, so equal cells stay on one side); a part with no
 * samples is cut evenly.  boxes: HOST int32 [px*py*pz, 6], box (a, b, c) at index
 * (a*py + b)*pz + c.  The same samples give the same boxes on every process.  Host only.
 * Errors: INVALID_ARG (n < 0, px, py or pz < 1, more than 1024 boxes, a cell outside
 * [0, 2^21)). */
int greem_domain_boxes(const int32_t *cells, int64_t n, int px, int py, int pz, int32_t *boxes);

/* The finest cells (reading of the Morton key: wrap into [0, L), floor((x/L) 2^21) clamped
 * to 2^21 - 1) of the particles idx[0..n) of pos [N, 3] (all device; idx NULL = the first n
 * particles): cells DEVICE int32 [n, 3].  Waits for the stream.  Errors: INVALID_ARG (bad
 * sizes, L <= 0, an index outside [0, N), a NaN/Inf coordinate), CUDA. */
int greem_cell_index(greem_ctx *ctx, const double *pos, int64_t N, double L, const int64_t *idx, int64_t n,
                     int32_t *cells);

/* Particles packed by destination domain for their redistribution (Sec. 2.2 step 7): each
 * particle's domain is the box (HOST boxes [ndom, 6]) holding its finest cell; pos_out
 * (wrapped into [0, L)), mass_out and ids_out (ids[i], or i when ids is NULL) receive the
 * particles of domain 0, then 1, ..., each in input order (stable); counts (HOST int64
 * [ndom]) gets the number per domain.  All arrays but boxes and counts are DEVICE, N rows,
 * owned by the caller.  Waits for the stream.  Errors: INVALID_ARG (bad sizes, boxes out of
 * range, a particle in no box or with a NaN/Inf coordinate), CUDA, OOM. */
int greem_domain_pack(greem_ctx *ctx, const double *pos, const float *mass, const int64_t *ids, int64_t N, double L,
                      const int32_t *boxes, int ndom, int64_t *counts, double *pos_out, float *mass_out,
                      int64_t *ids_out);

/* The local essential trees (Sec. 2.2 step 3; Eq. 10) of the tree built by the last
 * greem_build_tree (or force) call of this context, one box, for every domain d != self
 * of boxes (HOST [ndom, 6]): in node preorder, each accepted node as one item (its centre
 * of mass and mass) and the particles of each opened leaf that lie within r_cut of domain
 * d.  A node is visited when every ancestor was opened; it is pruned when its cell lies
 * farther than r_cut from the box (reading C2, the box in place of the group's particle
 * box), accepted when its level is at least l_min and the squared distance from its cell
 * centre to the nearest point of the box passes the opening test of the build's theta
 * (reading C1, or Eq. 12 when the build used it), and opened otherwise.  Items go out
 * packed by domain: pos_out DEVICE float64 [cap, 3] (absolute, wrapped), mass_out DEVICE
 * float32 [cap], ref_out DEVICE int64 [cap] or NULL (the sorted particle index, or
 * -1 - node for a node); counts HOST int64 [ndom] (0 for self and empty boxes); *total =
 * the items needed.  Each item is 28 bytes (Eq. 10 counts 16; the positions stay FP64
 * because the receiving process subtracts its group centres in FP64, Sec. 3.1.1).  At
 * theta = 0 no node is accepted and the items are exactly the particles within r_cut.
 * Waits for the stream.  Errors: INVALID_ARG (no tree, a multi-box call, bad boxes,
 * self >= ndom), CAPACITY (*total > cap: nothing past cap is written; call again with
 * cap >= *total), CUDA, OOM. */
int greem_let_export(greem_ctx *ctx, const int32_t *boxes, int ndom, int self, int64_t *counts, double *pos_out,
                     float *mass_out, int64_t *ref_out, int64_t cap, int64_t *total);

/* ---- Time integration (Sec. 2.2 steps 1, 6, 7; Sec. 2.4) --------------------------------
 * The paper kicks the velocities with the PM and then the PP force of the step (it keeps
 * no accelerations) and then drifts the positions; with the total force of one call that
 * is one kick and one drift per step (leapfrog with velocities half a step apart).
 * Comoving coordinates: with the momentum-like velocity w = a^2 dx/dt and the acceleration
 * of the comoving positions, the factors are f_kick = int dt/a and f_drift = int dt/a^2
 * over the step (greem_cosmo_factors); a non-cosmological run passes dt for both. */

/* v += f_kick * acc, per component in FP32 (vel, acc: float32 [N,3] device).  Errors:
 * INVALID_ARG (N < 1, NULL, non-finite f_kick), CUDA. */
int greem_kick(greem_ctx *ctx, float *vel, const float *acc, int64_t N, double f_kick);

/* pos += f_drift * vel in FP64, each coordinate wrapped into [0, L) by the key's wrap rule
 * (pos: float64 [N,3] device, updated in place; vel: float32 [N,3] device).  Errors:
 * INVALID_ARG (N < 1, NULL, L <= 0, non-finite f_drift), CUDA. */
int greem_drift(greem_ctx *ctx, double *pos, const float *vel, int64_t N, double L, double f_drift);

/* Shared adaptive timestep, Eq. 7: *dt = zeta * min_i( sqrt(eps/|a_i|), eps/|v_i| ),
 * computed as zeta * min( sqrt(eps / max|a|), eps / max|v| ) from device maxima of |a|^2
 * and |v|^2 in FP32 ((x^2 + y^2) + z^2); a term whose maximum is 0 gives no bound (+inf
 * when both are).  Waits for the stream.  Errors: INVALID_ARG (N < 1, NULL, eps <= 0,
 * zeta <= 0), CUDA. */
int greem_timestep(greem_ctx *ctx, const float *vel, const float *acc, int64_t N, double eps, double zeta,
                   double *dt);

/* Shared softening, Eq. 6, read as the physical softening: (1+z_crit)/(1+z) eps_fin for
 * z >= z_crit (then eps_fin (1+z_crit) in comoving coordinates, a constant), eps_fin for
 * z < z_crit (constant physically).  The force calls take comoving lengths: pass
 * greem_softening(...) * (1+z) as eps.  Host only. */
double greem_softening(double eps_fin, double z_crit, double z);

/* Comoving kick and drift factors of a step from scale factor a0 to a1 > a0 > 0 with
 * H(a) = H0 sqrt(omega_m a^-3 + (1 - omega_m - omega_l) a^-2 + omega_l): *kick = int da /
 * (a^2 H), *drift = int da / (a^3 H), by 4-point Gauss-Legendre on 4096 intervals.  Host
 * only.  Errors: INVALID_ARG (a0 <= 0, a1 <= a0, H0 <= 0, H^2 <= 0 on the interval). */
int greem_cosmo_factors(double a0, double a1, double omega_m, double omega_l, double h0, double *kick,
                        double *drift);

/* Measured arithmetic rates of this GPU at whatever clock it runs at the time: which = 0
 * FP32 FMA and 1 FP64 FMA (*tflops = 2 flops per FMA of an FMA-chain microbenchmark over
 * all SMs); 2 the force kernel's own packed pair loop over list entries held in shared
 * memory, with no list streaming or group overhead (42 flops per pair): the ceiling of
 * this formulation of Eq. 1-2.  Errors: INVALID_ARG, CUDA. */
int greem_peak_tflops(greem_ctx *ctx, int which, double *tflops);

const char *greem_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GREEM_H */
