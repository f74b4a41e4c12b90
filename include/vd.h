/*
 * vd.h — C ABI of libvd: GPU detection of topological changes in dynamic
 * centroidal Voronoi diagrams of lattice bubbles (M. Bernaschi, M. Lulli,
 * M. Sbragaglia, "GPU Based Detection of Topological Changes in Voronoi
 * Diagrams", arXiv:1607.00908).
 *
 * One frame of a periodic 2D scalar field goes through, on the GPU:
 *   threshold -> periodic connected-component labels     (Section 3.1)
 *   -> 1/1024-site centre of mass per bubble             (Section 3.1)
 *   -> exact digital Voronoi colouring of every site     (Section 3.2.1)
 *   -> Delaunay links from owner changes                 (Section 3.2.2)
 *   -> label isomorphism with the previous frame         (Section 3.2.3)
 *   -> breaking / arising links, local and global trigger (Sections 3.2.3-3.2.4)
 * All arithmetic is integer; results are bit-exact and deterministic.
 *
 * Conventions shared by every call:
 *  - Every function returns vd_status (0 = VD_OK, negative = error). No C++
 *    exception crosses this boundary.
 *  - Fields are float32, row-major, Ly rows of Lx values, row stride `pitch`
 *    in elements (pitch >= Lx), periodic in both axes.
 *  - Labels are int32 in 0..K-1: the rank of the bubble's smallest linear
 *    index y*Lx + x; background is -1.
 *  - Centroids are int32 pairs (cx, cy) in 1/1024 site, in [0, 1024*L).
 *  - An edge/link key is uint64 (lo << 32) | hi with lo < hi labels.
 *  - Device work is asynchronous on the stream given at creation. Getters
 *    synchronise that stream and copy into caller buffers, which may be host
 *    or device memory (cudaMemcpyDefault). After a push, the first state or
 *    change query copies every instance's counts (and, for changes, every
 *    instance's change lists, packed on the device) to the host at once;
 *    further queries about the same push are answered from those copies.
 *  - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef VD_H_
#define VD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vd_status;
enum {
    VD_OK = 0,
    VD_ERR_INVALID = -1,   /* bad argument, handle or configuration */
    VD_ERR_OOM = -2,       /* device allocation failed */
    VD_ERR_CAPACITY = -3,  /* a caller buffer or a device capacity was too small; counts are filled in */
    VD_ERR_CUDA = -4,      /* a CUDA runtime call failed */
    VD_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    VD_ERR_STATE = -6,     /* call out of order (e.g. results before any frame) */
    VD_ERR_UNSUPPORTED = -7,
    VD_ERR_BOUNDS = -8     /* checked build only: an index check failed (the access was skipped) */
};

/* Polarity of the spin variable of Section 3.1: a site is in a bubble when
 * value > threshold (VD_ABOVE) or value < threshold (VD_BELOW, the paper's
 * density convention). NaN is never in a bubble. */
enum { VD_ABOVE = 1, VD_BELOW = -1 };

typedef struct vd_config {
    int32_t Lx, Ly;            /* lattice size, 1 <= Lx, Ly, Lx*Ly < 2^31 */
    float threshold;           /* bubble threshold */
    int32_t polarity;          /* VD_ABOVE or VD_BELOW */
    int32_t connectivity;      /* 4 (default) or 8 neighbours (Section 3.1) */
    int32_t max_components;    /* capacity for bubbles per frame; 0 = ceil(Lx*Ly/2) (cannot overflow) */
    int32_t max_edges;         /* capacity for links per frame; 0 = 3*max_components + 64 */
    void* stream;              /* cudaStream_t for all device work; NULL = legacy default stream */
    int32_t events;            /* 1: classify the active labels into bulk / boundary events (Section 3.2.4) */
    int32_t match_rule;        /* VD_MATCH_OVERLAP (default) or VD_MATCH_CENTROID (Section 3.2.3) */
    int32_t match_radius;      /* VD_MATCH_CENTROID: largest centre displacement matched, in sites (>= 1) */
    int32_t edge_rule;         /* VD_EDGE_ADJ4 (default) or VD_EDGE_VERTEX (Section 3.2.2) */
    int32_t walls;             /* VD_WALL_X | VD_WALL_Y: bounded axes (0 = periodic torus) */
} vd_config;

/* Walls (the paper's channel geometry, Sections 3.2.1-3.2.2): a bounded axis
 * joins nothing across its ends -- no bubble, no minimum image, no link. The
 * library runs a bounded axis of length L as a periodic axis of length 2L
 * whose second half is never a bubble: every distance between two points of
 * the domain is then the plain one (below half the period). Obstacle sites
 * (vd_set_obstacles) are never in a bubble; their owner is VD_OWNER_OBSTACLE
 * (the paper's MAXLINK colour) and no link touches them. */
enum { VD_WALL_X = 1, VD_WALL_Y = 2 };
enum { VD_OWNER_OBSTACLE = -2 };

/* Links of the digital Voronoi diagram (Section 3.2.2). ADJ4: owners that
 * differ between +x / +y neighbouring sites, plus the exact incircle diagonal
 * of every plaquette with four distinct owners. VERTEX: the paper's own rule,
 * read at vertex sites only (three or more colour changes around the 8-site
 * frame) with its first- and second-neighbour conditions; the inner-frame
 * point of a diagonal is read as the plaquette centre, and its colour is its
 * Voronoi colour (the nearest centre over all centres, exact, ties to the
 * smallest label), as for every point of the stencil. The figure defining the
 * inner frame is lost, so the VERTEX rule follows that reading. */
enum { VD_EDGE_ADJ4 = 0, VD_EDGE_VERTEX = 1 };

/* Isomorphism Phi between past and now labels (Section 3.2.3). OVERLAP: the
 * mutual best overlap of the two frames' bubbles (largest shared site count,
 * ties to the smallest label). CENTROID: the paper's kinematic comparison of
 * the two sets of centres -- mutual nearest centres (minimum-image squared
 * distance in 1/1024 sites, ties to the smallest label) no farther apart than
 * match_radius sites. */
enum { VD_MATCH_OVERLAP = 0, VD_MATCH_CENTROID = 1 };

/* Fill `cfg` with defaults for an Lx x Ly lattice (threshold 0.5, VD_ABOVE,
 * 4-connectivity, automatic capacities, default stream, no event classes,
 * overlap match). */
vd_status vd_config_init(vd_config* cfg, int32_t Lx, int32_t Ly);

typedef struct vd_ctx vd_ctx;

/* Create a detector for one periodic lattice. Allocates all resident device
 * state (two label frames, centroids, links, scratch) on the current device.
 * `*out` is set on success. Errors: VD_ERR_INVALID (bad cfg), VD_ERR_OOM. */
vd_status vd_create(const vd_config* cfg, vd_ctx** out);

/* Enqueue one frame (Sections 3.1-3.2.4). `d_field` is a device pointer to
 * Ly rows of `pitch` floats; it must stay valid until the stream reaches
 * this work. The previous frame's labels and links stay resident on the
 * device; the first frame after creation reports no changes. Asynchronous:
 * device-side capacity overflows are reported by the next getter. */
vd_status vd_push_frame(vd_ctx* ctx, const float* d_field, size_t pitch);

/* Obstacle sites of the lattice: host array of Ly rows of `pitch` bytes, a
 * nonzero byte marks an obstacle (Lx <= pitch). Applies from the next pushed
 * frame on; the mask stays until it is replaced (an all-zero mask clears it).
 * Errors: VD_ERR_INVALID, VD_ERR_CUDA. */
vd_status vd_set_obstacles(vd_ctx* ctx, const uint8_t* h_mask, int64_t pitch);

/* Same as vd_push_frame with a host-memory field: copies it to a context-owned
 * device buffer on the context stream first (synchronous w.r.t. `h_field`). */
vd_status vd_push_frame_host(vd_ctx* ctx, const float* h_field, size_t pitch);

/* Result of the last pushed frame (Sections 3.2.3-3.2.4). The caller owns the
 * arrays and states their capacities; the library always fills the counts and
 * writes an array only when it fits (else returns VD_ERR_CAPACITY after
 * writing all counts). `breaking` / `breaking_prev` / `arising` are sorted by
 * now-key; `breaking_prev[i]` is breaking[i] in past labels. `active` (length
 * n_now) holds per-label flags: bit 0 (VD_EV_ACTIVE) is the local trigger, set
 * for labels at an end of a flip; the event classes of Section 3.2.4
 * ("Extracting Topology Change Events") sit above it: VD_EV_BULK (active and
 * linked to at least three active labels in the past or in the now
 * triangulation), VD_EV_BOUNDARY (active, a boundary point of one
 * triangulation -- an end of a link whose ends share exactly one neighbour --
 * linked there to an active boundary point), VD_EV_BPOINT_NOW /
 * VD_EV_BPOINT_PAST (the active label is a boundary point of that
 * triangulation); the classes are computed when the config sets `events`.
 * Inactive labels are 0. */
enum { VD_EV_ACTIVE = 1, VD_EV_BULK = 2, VD_EV_BOUNDARY = 4, VD_EV_BPOINT_NOW = 8, VD_EV_BPOINT_PAST = 16 };
typedef struct vd_changes {
    int64_t frame_index;       /* 0-based index of the frame these results belong to */
    int32_t n_prev, n_now;     /* bubbles in the past and current frame */
    int32_t n_matched;         /* labels matched by the isomorphism */
    int32_t n_edges;           /* links of the current frame */
    int32_t n_breaking, n_arising;
    int32_t global_trigger;    /* 1 when n_breaking + n_arising > 0 */
    uint64_t* breaking;        int32_t cap_breaking;
    uint64_t* breaking_prev;   /* same capacity as breaking; may be NULL */
    uint64_t* arising;         int32_t cap_arising;
    uint8_t* active;           int32_t cap_active;   /* may be NULL */
} vd_changes;

vd_status vd_get_changes(vd_ctx* ctx, vd_changes* out);

/* Parity/introspection getters for the last pushed frame. Each copies into a
 * caller buffer (host or device) of `cap` elements and sets the element count
 * in *n; VD_ERR_CAPACITY (buffer untouched) when cap is too small. */
vd_status vd_get_counts(vd_ctx* ctx, int32_t* K, int32_t* n_edges, int64_t* frame_index);
vd_status vd_get_labels(vd_ctx* ctx, int32_t* out, int64_t cap, int64_t* n);        /* Ly*Lx, row-major */
vd_status vd_get_centroids_q10(vd_ctx* ctx, int32_t* out, int64_t cap, int64_t* n); /* K pairs (cx, cy): cap counts int32 */
vd_status vd_get_owners(vd_ctx* ctx, int32_t* out, int64_t cap, int64_t* n);        /* Ly*Lx Voronoi owners */
vd_status vd_get_edges(vd_ctx* ctx, uint64_t* out, int64_t cap, int64_t* n);        /* sorted unique keys */
vd_status vd_get_match(vd_ctx* ctx, int32_t* phi, int64_t cap, int64_t* n);         /* K_prev entries, -1 = unmatched */

/* Tuning of the launch shapes (not part of the result: every setting gives
 * bit-identical output). voronoi_patch: the patch layout of the owner kernel,
 * which splits each 64 x 32 tile into patches that keep their own candidate
 * centres (VD_PATCH_8x8, the default, 16x8, 32x8 or 16x16 sites); bucket_pct:
 * side of the centre bucket grid in percent of the mean centre spacing
 * (25..400, default 100); ring0: sites beyond the tile reached by the first
 * round of the owner search (0..256, default 9); graph_blocks: the graph stage
 * (CSR, match, flips) as one block per instance in two launches (1) or as a
 * chain of grid-wide launches over all instances' rows and links, with the
 * match on a second stream beside the owner, link and CSR kernels (0, the
 * default). Applies from the next push;
 * synchronises the stream. The autotuner (paper_1607_00908_gb300/autotune.py)
 * times candidates and keeps the fastest per lattice-size and density class. */
enum { VD_PATCH_8x8 = 0, VD_PATCH_16x8 = 1, VD_PATCH_32x8 = 2, VD_PATCH_16x16 = 3 };
typedef struct vd_tuning {
    int32_t voronoi_patch;
    int32_t bucket_pct;
    int32_t ring0;
    int32_t graph_blocks;
} vd_tuning;
vd_status vd_set_tuning(vd_ctx* ctx, const vd_tuning* t);
vd_status vd_get_tuning(vd_ctx* ctx, vd_tuning* t);

/* Checkpoint / resume. Section 3.2.3 compares every frame with the previous
 * one, so the state a context carries from frame to frame is that frame's
 * labels (foreground bits and per-run labels), Q10 centroids with their
 * bucket grid, its links (sorted adjacency rows of both directions) and the
 * frame count. vd_export_state copies it into a caller-owned HOST buffer of
 * `cap` bytes and sets *n_bytes to the size needed (VD_ERR_CAPACITY, nothing
 * written, when buf is NULL or too small). vd_import_state replaces a
 * context's last frame by an exported state: the next push compares against
 * it, so a context resumed from a checkpoint reports bit-identical changes
 * to the uninterrupted one. The blob (versioned, native byte order, with a
 * checksum) must come from a lattice of the same size and walls and fit the
 * context's capacities; options (threshold, polarity, rules) are taken from
 * the importing context, and obstacle masks are configuration, set again with
 * vd_set_obstacles. Every value is range-checked before anything reaches the
 * device: a damaged or foreign blob gives VD_ERR_INVALID and leaves the
 * context unchanged. After an import, labels, centroids, links and counts
 * describe the imported frame; owners, the match and the changes are not part
 * of the state (VD_ERR_STATE until the next push). Both calls synchronise the
 * context's stream. Export errors: VD_ERR_STATE (no frame yet), the status of
 * a failed last frame, VD_ERR_CAPACITY, VD_ERR_CUDA; a frame-sequence batch
 * gives VD_ERR_UNSUPPORTED (its frames are not independent lattices). */
vd_status vd_export_state(vd_ctx* ctx, void* buf, int64_t cap, int64_t* n_bytes);
vd_status vd_import_state(vd_ctx* ctx, const void* buf, int64_t n_bytes);

/* Stage timing (measurement support, not part of the detect result). When
 * enabled, every vd_push_frame records CUDA events on the context stream at
 * the boundaries of the pipeline stages (labelling tiles, bubble merge and
 * centroids, run labels and overlaps, Voronoi owners, links,
 * adjacency/match/flips) and runs
 * without graph replay. vd_get_timing synchronises the stream and returns
 * the summed milliseconds per stage since the last call (stage_ms has cap
 * entries; *n_stages is set), the number of kernels launched and frames
 * pushed since creation. Names via vd_stage_name. */
vd_status vd_set_timing(vd_ctx* ctx, int32_t enable);
vd_status vd_get_timing(vd_ctx* ctx, double* stage_ms, int32_t cap, int32_t* n_stages,
                        int64_t* n_kernel_launches, int64_t* n_frames);
const char* vd_stage_name(int32_t stage);

/* Test support for the bounded device wait (not part of the detect result).
 * The only device-side wait of a step is the decoupled look-back of its
 * prefix scans: a scan tile waits for its predecessors' flags and gives up
 * after a bounded number of polls (2^20 by default). A tile that gives up
 * sums its prefix directly from every earlier item (slow, but no offset is
 * ever wrong and the tiles after it proceed), and the frame then reports
 * VD_ERR_TIMEOUT from every getter; the context stays usable and the next
 * frame starts without a past frame. This call makes tile `tile` of scan
 * `kind` (0 = the bubble-rank scan, the first scan of a step; 1 buckets,
 * 2 link degrees, 3-4 flip counts) withhold its flag in every following push,
 * so that its successor's wait runs out after `spin_limit` polls (0 = the
 * default limit). tile = -1 turns the hold off. Synchronous; errors:
 * VD_ERR_INVALID, VD_ERR_CUDA. */
vd_status vd_debug_hold_scan_flag(vd_ctx* ctx, int32_t kind, int64_t tile, int32_t spin_limit);

/* Checked build. The same sources compiled with -DVD_CHECKED give
 * libvd_checked.so (built beside libvd.so), which tests the index of every
 * scatter access whose index is computed from data (piece ids, run slots,
 * bucket cells and positions, overlap and link list positions, queue
 * positions, owner writes, CSR columns, flip lists, scan offsets) against
 * its array before the access. A failed test skips the access, records the
 * check's id and the index (the first of the step is kept) and makes every
 * getter of that step return VD_ERR_BOUNDS. It stands in for a memory
 * checker where none can run. In the regular build the tests compile away.
 * vd_debug_check_info synchronises the stream and returns *checked = 1 in
 * the checked build (0 otherwise), the id of the first failed check of the
 * last step (0 = none; ids 1..20 name the checked accesses) and its index.
 * vd_debug_force_check(id) makes check `id` fail from the next push on,
 * without any access (the test of the reporting path); 0 turns it off; no
 * effect in the regular build. Errors: VD_ERR_INVALID, VD_ERR_CUDA. */
vd_status vd_debug_check_info(vd_ctx* ctx, int32_t* checked, int32_t* first_check, int64_t* index);
vd_status vd_debug_force_check(vd_ctx* ctx, int32_t id);

/* Release all device state of the context (waits for its stream first). */
vd_status vd_destroy(vd_ctx* ctx);

/* Voronoi owners without any device allocation. The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc
 * (processes whose device memory all belongs to another framework's
 * allocator, real-time or embedded hosts that allocate everything at
 * start-up and may not allocate afterwards). It computes the same exact colouring as the pipeline's owner
 * step: owner(x,y) = the label i minimising |1024*(x,y) - c_i|^2 (minimum
 * image, ties to the smallest i), or -1 when K == 0.
 *   d_centroids_q10  device, K pairs (cx, cy) in 1/1024 site, in [0, 1024*L);
 *                    pairs outside that range are ignored
 *   d_owners         device, Ly*Lx int32, row-major (written)
 *   stream           cudaStream_t (NULL = legacy default stream)
 * Its scratch is one static __device__ array of about 1.5 MB per GPU, held
 * until the process exits: at most 65536 centroids and 65536 bucket cells
 * per call (larger K returns VD_ERR_CAPACITY without launching anything).
 * Every call shares that array: calls whose device work may overlap (other
 * streams, other host threads) race and must be serialised by the caller.
 * The first call on a device resolves the array's device address (a runtime
 * query, no allocation); make that first call before any stream capture. A
 * device reset (cudaDeviceReset) invalidates the resolved address: do not
 * use this entry point across a reset. Asynchronous on `stream`; each launch
 * is checked as it is enqueued; errors: VD_ERR_INVALID, VD_ERR_CAPACITY,
 * VD_ERR_CUDA. */
vd_status vd_voronoi_owners_static(const int32_t* d_centroids_q10, int32_t K, int32_t Lx, int32_t Ly,
                                   int32_t* d_owners, void* stream);

/* Static description of a status code. */
const char* vd_status_string(vd_status s);

/* ---------------------------------------------------------------------------
 * Batched form: many independent lattices of uneven size advance one frame
 * per vd_batch_push. Every pipeline stage runs as one launch over all
 * instances (work lists of (instance, tile)); the sequence is captured once
 * into a CUDA graph and replayed.
 * ------------------------------------------------------------------------- */
typedef struct vd_batch vd_batch;
/* the checked-build calls (see vd_debug_check_info) for a batch */
vd_status vd_batch_debug_check_info(vd_batch* b, int32_t* checked, int32_t* first_check, int64_t* index);
vd_status vd_batch_debug_force_check(vd_batch* b, int32_t id);

/* `cfgs[i]` describes instance i; all share cfgs[0].stream. */
vd_status vd_batch_create(const vd_config* cfgs, int32_t n, vd_batch** out);
/* Frame sequence of one lattice as a batch: the n instances are n
 * consecutive frames of the same field. Instance i's past frame is instance
 * i-1 of the same vd_batch_push (instance 0's is instance n-1 of the
 * previous push), so each push advances the sequence by n frames with every
 * stage launched once for all of them (Sections 3.1-3.2.4 per frame, as in
 * vd_push_frame). Getters take the frame's position 0..n-1 in the last push;
 * vd_changes.frame_index counts frames since creation. */
vd_status vd_batch_create_sequence(const vd_config* cfg, int32_t n_frames, vd_batch** out);
/* `d_fields` is a HOST array of n device pointers (each Ly*pitch floats,
 * pitch = Lx); instance i reads d_fields[i]. Enqueues one step. */
vd_status vd_batch_push(vd_batch* b, const float* const* d_fields);
/* Same with HOST fields (h_fields[i]: Ly*Lx floats, row-major): equivalent to
 * vd_batch_stage_host followed by vd_batch_push_staged (below). Pinned host
 * memory makes the copies asynchronous; the caller keeps the host arrays
 * unchanged until the step has been queried. */
vd_status vd_batch_push_host(vd_batch* b, const float* const* h_fields);
/* Advance only the `n_active` instances listed in `active` (host array of
 * instance ids, each at most once); the others keep their state. */
vd_status vd_batch_push_subset(vd_batch* b, const int32_t* active, int32_t n_active,
                               const float* const* d_fields);
vd_status vd_batch_get_changes(vd_batch* b, int32_t i, vd_changes* out);

/* Obstacle sites of instance i (see vd_set_obstacles). */
vd_status vd_batch_set_obstacles(vd_batch* b, int32_t i, const uint8_t* h_mask, int64_t pitch);

/* Double-buffered host input. vd_batch_stage_host copies h_fields (HOST array
 * of n HOST pointers, Ly*Lx floats each, pinned for asynchrony) into the next
 * of two batch-owned input buffers on a copy stream of the batch and returns;
 * the copy waits only for the step that last read that buffer. It does not
 * advance the batch. vd_batch_push_staged enqueues one step on the most
 * recently staged inputs (the step waits for their copy); VD_ERR_STATE if
 * nothing was staged since the last vd_batch_push_staged. Staging the next
 * frames before querying the current step's results overlaps the host->device
 * copy with the step. The caller keeps the host arrays unchanged until the
 * step that reads them has been queried. */
vd_status vd_batch_stage_host(vd_batch* b, const float* const* h_fields);
vd_status vd_batch_push_staged(vd_batch* b);

/* Results of every instance of the last push in one call. Per-instance arrays
 * (n entries, may be NULL) receive the counts and a status per instance (the
 * vd_status its vd_batch_get_changes would return; failed instances add no
 * entries). The change lists of all instances are packed instance-major into
 * the list arrays (may be NULL); the totals are always set. VD_ERR_CAPACITY
 * when a non-NULL list array is smaller than its total (nothing is copied into
 * the lists then). */
typedef struct vd_batch_changes {
    int32_t* status;
    int32_t* n_prev;
    int32_t* n_now;
    int32_t* n_breaking;
    int32_t* n_arising;
    uint64_t* breaking;        /* all instances' breaking keys */
    uint64_t* breaking_prev;   /* their past keys, same order */
    int64_t cap_breaking;
    uint64_t* arising;         int64_t cap_arising;
    uint8_t* active;           int64_t cap_active;   /* K entries per instance */
    int64_t total_breaking, total_arising, total_active;   /* set by the call */
} vd_batch_changes;
vd_status vd_batch_get_changes_all(vd_batch* b, vd_batch_changes* out);
vd_status vd_batch_get_labels(vd_batch* b, int32_t i, int32_t* out, int64_t cap, int64_t* n);
vd_status vd_batch_get_owners(vd_batch* b, int32_t i, int32_t* out, int64_t cap, int64_t* n);
vd_status vd_batch_get_edges(vd_batch* b, int32_t i, uint64_t* out, int64_t cap, int64_t* n);
vd_status vd_batch_get_centroids_q10(vd_batch* b, int32_t i, int32_t* out, int64_t cap, int64_t* n);
vd_status vd_batch_get_counts(vd_batch* b, int32_t i, int32_t* K, int32_t* n_edges, int64_t* frame_index);
/* Tuning of a batch (as vd_set_tuning; one setting for all instances). */
vd_status vd_batch_set_tuning(vd_batch* b, const vd_tuning* t);
vd_status vd_batch_get_tuning(vd_batch* b, vd_tuning* t);
/* Checkpoint / resume of instance i of an independent batch (as
 * vd_export_state / vd_import_state). */
vd_status vd_batch_export_state(vd_batch* b, int32_t i, void* buf, int64_t cap, int64_t* n_bytes);
vd_status vd_batch_import_state(vd_batch* b, int32_t i, const void* buf, int64_t n_bytes);
/* Stage timing of a batch (as vd_set_timing / vd_get_timing; *n_steps
 * counts pushes). */
vd_status vd_batch_set_timing(vd_batch* b, int32_t enable);
vd_status vd_batch_get_timing(vd_batch* b, double* stage_ms, int32_t cap, int32_t* n_stages,
                              int64_t* n_kernel_launches, int64_t* n_steps);
vd_status vd_batch_destroy(vd_batch* b);

/* ---------------------------------------------------------------------------
 * Served form: frames of many simulations arrive over time; continuous
 * batching (the paper runs its detection inside a running simulation every
 * few steps, Section 4; a server does so for many simulations at once). The
 * server keeps every simulation's state resident (one batch instance per
 * simulation) and runs steps over the simulations that have a waiting frame:
 * at most one frame per simulation per step, at most max_batch simulations,
 * oldest arrival first, admitted only while the resident state plus the
 * frames in flight fit hbm_budget_bytes. Two steps are kept queued on the
 * device, so frames that arrive while a step runs join the next one.
 * Simulations can be opened and closed while others run.
 * ------------------------------------------------------------------------- */
typedef struct vd_server vd_server;
typedef struct vd_server_done {
    int64_t ticket;             /* from vd_server_submit */
    int32_t sim;
    int32_t status;             /* VD_OK or the frame's device error */
    int64_t t_arrival_ns;       /* the frame's arrival time given to vd_server_submit */
    int64_t t_submit_ns;        /* when vd_server_submit was called (vd_server_clock_ns clock) */
    int64_t t_done_ns;          /* when vd_server_poll saw the step finish */
    int32_t n_bubbles, n_edges, n_breaking, n_arising;
} vd_server_done;

/* A server whose device work runs on `stream` (cudaStream_t; the configs'
 * own stream fields are ignored), opening the `n_sims` simulations of `sims`
 * (n_sims may be 0). Allocates their resident state; VD_ERR_CAPACITY when it
 * alone exceeds the budget. */
vd_status vd_server_create(const vd_config* sims, int32_t n_sims, int64_t hbm_budget_bytes, int32_t max_batch,
                           void* stream, vd_server** out);
/* Open one more simulation while others run; *sim receives its id. Its
 * resident state is allocated now and admitted only if every open
 * simulation's state still fits the budget (VD_ERR_CAPACITY otherwise,
 * nothing kept). */
vd_status vd_server_open_sim(vd_server* sv, const vd_config* cfg, int32_t* sim);
/* Close a simulation with no frame queued or in flight (VD_ERR_STATE
 * otherwise); its id is not reused. Its state leaves the budget once every
 * simulation opened together with it is closed. */
vd_status vd_server_close_sim(vd_server* sv, int32_t sim);
/* The host steady clock of the server's timestamps, in ns. */
vd_status vd_server_clock_ns(int64_t* t);
/* Queue one frame (device pointer, Ly*Lx floats) of simulation `sim` that
 * arrived at t_arrival_ns (vd_server_clock_ns clock; <= 0: now). Latency is
 * counted from the arrival, so host delay before the submit is included. The
 * caller keeps the frame valid until it is reported done. */
vd_status vd_server_submit(vd_server* sv, int32_t sim, const float* d_field, int64_t t_arrival_ns, int64_t* ticket);
/* Run the scheduler: retire finished steps (filling `done`, up to cap
 * entries) and launch new steps. wait != 0 blocks until at least one frame
 * finishes or nothing is in flight. */
vd_status vd_server_poll(vd_server* sv, int32_t wait, vd_server_done* done, int32_t cap, int32_t* n_done);
/* With keep != 0, every poll also copies the breaking / arising lists and
 * active flags of each frame it retires to host memory (one gather per
 * group of simulations, on a side stream, before any of those simulations
 * is given its next frame); vd_server_get_frame_changes returns them by
 * ticket until the next poll. Off by default. */
vd_status vd_server_keep_changes(vd_server* sv, int32_t keep);
/* Changes of a frame retired by the most recent vd_server_poll (as
 * vd_get_changes); VD_ERR_STATE for any other ticket or when changes are not
 * kept. */
vd_status vd_server_get_frame_changes(vd_server* sv, int64_t ticket, vd_changes* out);
/* Results of a simulation's last finished frame; VD_ERR_STATE while one of
 * its frames is in flight. */
vd_status vd_server_get_changes(vd_server* sv, int32_t sim, vd_changes* out);
vd_status vd_server_get_labels(vd_server* sv, int32_t sim, int32_t* out, int64_t cap, int64_t* n);
/* Checkpoint / resume of one simulation (as vd_export_state /
 * vd_import_state); VD_ERR_STATE while it has a frame in flight (or, for
 * import, queued). */
vd_status vd_server_export_state(vd_server* sv, int32_t sim, void* buf, int64_t cap, int64_t* n_bytes);
vd_status vd_server_import_state(vd_server* sv, int32_t sim, const void* buf, int64_t n_bytes);
vd_status vd_server_stats(vd_server* sv, int64_t* steps, int64_t* frames_done, int64_t* resident_bytes,
                          int64_t* queued);
vd_status vd_server_destroy(vd_server* sv);

#ifdef __cplusplus
}
#endif
#endif /* VD_H_ */
