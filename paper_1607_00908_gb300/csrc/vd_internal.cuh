// Internal data structures and device helpers of libvd.
//
// Every context is a batch of independent lattices ("instances"); the plain
// single-lattice context is a batch of one. Per-instance arrays live in pooled
// device buffers at fixed per-instance offsets; per-frame scratch that holds
// a variable number of items (pieces of bubbles inside tiles) comes from one
// pool shared by all instances of a step. Kernels take a step table that maps
// their block or item index to (instance, local index).
#pragma once

#include <cuda_runtime.h>
#include <climits>
#include <stdint.h>

namespace vd {

// ---------------------------------------------------------------------------
// Tiling
// ---------------------------------------------------------------------------
constexpr int TW = 64;          // labelling tile width  (sites)
constexpr int TH = 32;          // labelling tile height (sites)
constexpr int TRUNS = TH * 32;  // run slots per labelling tile (at most 32 runs per 64-site row)
constexpr int TSITES = TW * TH; // 2048
constexpr int TTHREADS = 256;   // 8 threads per tile row, 8 sites each
constexpr int BORDER = 2 * (TW + TH);   // left col, right col, top row, bottom row

constexpr int VW = 32;          // Voronoi tile width
constexpr int VH = 32;          // Voronoi tile height
constexpr int VTHREADS = 256;

constexpr int Q = 1024;         // centroid fixed point: 1/1024 site

// Bubble ids are the ranks of the roots in raster order of their first sites.
// Roots are counted per root group (RGW consecutive bitmask words of one row,
// 32 * RGW sites); the groups are scanned and a root adds the bits before it
// in its own group.
constexpr int RGW = 8;

constexpr unsigned long long EMPTY_KEY = ~0ull;

// owners that are not bubbles: the site of an obstacle (the paper's MAXLINK
// colour) and a site beyond a wall (a bounded axis runs with twice its length)
constexpr int OWN_OBSTACLE = -2;
constexpr int OWN_OUTSIDE = -3;

// error bits in InstState::err and Globals::err
enum : int {
    ERR_EDGE_CAP = 1,       // link hash or list overflow
    ERR_OVL_CAP = 2,        // overlap hash overflow
    ERR_PIECE_CAP = 4,      // tile-piece pool overflow
    ERR_COMP_CAP = 8,       // more bubbles than max_components
    ERR_TIMEOUT = 16,       // bounded device wait expired
    ERR_FLIP_CAP = 32,
    ERR_PREV = 64,          // the past frame (same step) had an error
    ERR_BOUNDS = 128,       // an index check of the checked build failed
};

// bits of the per-bubble active flags: bit 0 is the local trigger (an end of a
// breaking or arising link); the others are the event classes of Section
// 3.2.4 (bulk / boundary event point; boundary point of the now / past
// triangulation)
enum EventBits : unsigned {
    EV_ACTIVE = 1u,
    EV_BULK = 2u,
    EV_BOUNDARY = 4u,
    EV_BPOINT_NOW = 8u,
    EV_BPOINT_PAST = 16u,
};

// ---------------------------------------------------------------------------
// Static per-instance description (written once at creation)
// ---------------------------------------------------------------------------
struct InstDesc {
    int Lx, Ly;
    float thr;
    int pol;
    int ntx, nty;            // labelling tiles
    int vtx, vty;            // Voronoi tiles
    int wpr;                 // 32-bit bitmask words per lattice row
    int seq_prev;            // instance holding this instance's past frame (itself when independent)
    int seq_same;            // 1: that past frame is produced in the same step (frame sequence)
    int gpr;                 // root groups per lattice row (RGW words each)
    long long site_off;      // labels / owners pools
    long long word_off;      // fg-bit / root-bit pools (Ly * wpr words)
    long long grp_off;       // root-group count / rank pools (Ly * gpr groups)
    long long tile_off;      // per-labelling-tile pools (tile piece base/count)
    long long border_off;    // border pool (ntx*nty*BORDER)
    long long comp_off;      // per-bubble pools (comp_cap entries, +1 for offsets)
    long long edge_off;      // per-link pools (edge_cap entries)
    long long ehash_off;     // link hash (ehash_mask+1 slots)
    long long ohash_off;     // overlap hash (ohash_mask+1 slots)
    long long bucket_off;    // bucket grid pools (bucket_cap+1)
    long long ovl_off;       // overlap occupancy list (ovl_cap)
    int comp_cap, edge_cap;
    int ehash_mask, ohash_mask;
    int bucket_cap, ovl_cap;
    int events;              // classify the active labels (Section 3.2.4)
    int match_rule;          // VD_MATCH_OVERLAP / VD_MATCH_CENTROID
    int match_radius;        // centroid match: largest displacement, sites
    int conn8;               // 8-connectivity (else 4)
    int edge_rule;           // VD_EDGE_ADJ4 / VD_EDGE_VERTEX
    int masked;              // walls or obstacles: owners outside the domain / on obstacles are marked
    int uLx, uLy;            // the domain as the caller sees it; a bounded axis runs as 2 x its length
    // tuning (vd_batch_set_tuning): bucket side in percent of the mean centre
    // spacing; radius in sites of the first ring round of the owner search
    int bucket_pct;
    int ring0;
    int pad3;
};

// ---------------------------------------------------------------------------
// Dynamic per-instance state (device memory)
// ---------------------------------------------------------------------------
struct InstState {
    const float* field;      // this step's input
    long long pitch;
    int slot;                // buffer of this instance's last finished frame; this step writes slot ^ 1
    int has_prev;            // a past frame exists for this step
    int prev_inst;           // instance and buffer holding the past frame (set at step begin)
    int prev_buf;
    int prev_same;           // the past frame is written in this step (by another instance)
    int last_ok;             // the last finished frame had no device error
    int Kb[2];               // bubbles of the frame stored in each buffer
    int Eb[2];               // links of the frame stored in each buffer
    long long frame;         // index of the frame in progress / last finished
    int K, K_prev;           // bubbles now (clamped to the capacity) / previous frame
    int K_roots;             // roots found by labelling this step, before clamping
    int E, E_prev;           // links now / previous frame
    int B, nbx, nby;         // bucket grid of the frame in progress
    int Bs[2], nbxs[2], nbys[2];   // bucket grid of the frame stored in each buffer
    int n_matched;
    int n_break, n_arise;
    int n_wide;
    int n_ovl;               // overlap pairs this frame
    int n_edge_list;         // unique links inserted in the hash (= E)
    int n_eapp;              // links appended by Voronoi tiles (before dedup)
    int n_oapp;              // overlap pairs appended by label tiles (before merge)
    int err;
    int rep_K_prev;          // bubbles of the past frame used by the last step
    int pad1;
};

// per-step global counters
struct Globals {
    int n_pieces;
    int n_wide;
    int err;
    unsigned scan_step;      // bumped once per step; with the scan kind it tags look-back flags
    int scan_ticket[8];      // dynamic tile index of each scan kind (reset once per step)
    // test support (vd_debug_hold_scan_flag): tile dbg_tile - 1 of scan kind
    // dbg_kind never publishes its look-back flag (dbg_tile 0: no tile), and
    // look-back waits give up after dbg_spin polls when dbg_spin > 0
    int dbg_kind;
    int dbg_spin;
    long long dbg_tile;
    // checked build: the first failed index check of the step (id, index;
    // id 0: none) and the test hook that makes check dbg_chk fail
    int chk_id;
    int dbg_chk;
    long long chk_index;
    // instances whose link or overlap list overflowed: their hashes keep
    // unlisted keys, which the first kernel of their next step clears
    int lists_over;
};

// ---------------------------------------------------------------------------
// Device pools
// ---------------------------------------------------------------------------
struct Pools {
    InstDesc* desc;
    InstState* st;
    Globals* g;
    // sites
    int* owners;
    // bitmask words
    unsigned* fgbits[2];     // foreground bits of the frames in slot 0 / 1
    int* rp;                 // piece id of every run of this step's frames (tile run slots)
    int* rl[2];              // bubble label of every run of the frames in slot 0 / 1
    int* lab_out;            // per-site labels of one instance, expanded on request
    unsigned* rootbits;
    unsigned* obst;          // obstacle bits (word layout of the foreground bits)
    int* rgcnt;              // roots per root group (zero between steps)
    int* rankpre;            // exclusive rank prefix per root group (this step)
    // labelling tiles
    int* tile_pbase;         // first piece index of the tile in the piece pool
    int* tile_pcnt;          // number of pieces of the tile
    int* border;
    // pieces (bubble fragments inside one labelling tile)
    int piece_cap;
    int* p_q;                // linear index of the piece's first site
    int* p_inst;
    int* p_n;
    int* p_su;               // sum of (x - x_q) over the piece
    int* p_sv;               // sum of (y - y_q)
    int* p_parent;           // union-find over pieces (root = piece with smallest q)
    int* p_comp;             // bubble id (roots after ranking, every piece after k_comp_final)
    long long* p_accn;
    long long* p_accx;
    long long* p_accy;
    int* wide;               // pieces whose sums need the exact per-site path
    // bubbles
    int2* cq[2];             // centroids of the frame in each buffer (the step writes slot ^ 1)
    int* comp_root;          // root piece of each bubble
    int* bcnt;               // bucket counts (zero between steps)
    // bucket grid of the frame in each buffer: offsets (per-instance scan
    // values), centroids in bucket order, bubble ids in bucket order
    int* boff[2];
    int2* bcq[2];
    int* bid[2];
    unsigned long long* best_n;   // indexed by past label
    unsigned long long* best_p;   // indexed by now label
    int* phi;                // past -> now, -1 unmatched
    int* inv;                // now -> past
    unsigned char* active;
    int* deg;                // link degree counts (zero between steps)
    int* rowoff[2];          // CSR row offsets (per-instance scan values) of past/now frames
    int* tlen;               // length of the translated past row of each now-bubble
    int* fcnt;               // per-row flip counts: breaking, arising
    int* fcnt_a;
    int* foff;
    int* foff_a;
    // links
    // CSR of both directions (row a lists every neighbour of a, sorted):
    // 2 * edge_cap entries per instance from 2 * edge_off
    int* cols[2];            // past/now frames
    int* tcols;              // translated past rows, each at its past row's position
    unsigned long long* ehash;
    int* elist;              // occupied hash slots
    unsigned long long* ohash;
    unsigned* oval;
    int* olist;
    unsigned long long* brk;
    unsigned long long* brk_prev;
    unsigned long long* ari;
    unsigned long long* ekeys;   // per-tile unique links appended by the Voronoi pass; getter staging
    unsigned long long* oapp_key;   // per-tile (past, now) pairs appended by the label pass
    unsigned* oapp_cnt;
    // scan scratch
    unsigned long long* scan_flags;
    long long scan_flag_cap;     // tiles of SCAN_TILE elements
    // field pointers of this step (indexed by instance)
    const float* const* fields;
    const long long* pitches;
};

// Step table: which instances run this step and how blocks map onto them.
struct StepTable {
    int n_act;
    const int* act;              // instance ids
    const int* tileA_pre;        // prefix of labelling tiles over act (n_act+1)
    const int* tileV_pre;        // prefix of Voronoi tiles
    const long long* grp_pre;    // prefix of root groups
    // device-computed prefixes over act (n_act+1 each), filled by k_plan
    long long* pre;              // NPRE arrays back to back
};

enum PreIdx : int {
    PRE_K = 0,      // bubbles now
    PRE_KP,         // bubbles previous frame
    PRE_NB,         // buckets
    PRE_E,          // links now
    PRE_EP,         // links previous frame
    PRE_O,          // overlap pairs
    PRE_FB,         // breaking links
    PRE_FA,         // arising links
    PRE_EA,         // appended links
    PRE_OA,         // appended overlap pairs
    PRE_KR,         // roots found by labelling (bubbles before clamping to the capacity)
    NPRE
};
constexpr int PRE_ALL = (1 << NPRE) - 1;
__host__ __device__ constexpr int pre_bit(int k) { return 1 << k; }

__device__ __forceinline__ long long* pre_arr(const StepTable& T, int which) {
    return T.pre + (long long)which * (T.n_act + 1);
}

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline long long wrap_ll(long long d, long long L) {
    // minimum image in [-(L/2), L - L/2)
    long long h = L / 2;
    long long r = (d + h) % L;
    if (r < 0) r += L;
    return r - h;
}

__device__ __forceinline__ int upper_bound_int(const int* a, int n, int v) {
    // first index i in [0, n] with a[i] > v; a has n+1 entries nondecreasing
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int upper_bound_ll(const long long* a, int n, long long v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// map a virtual item index onto (slot in act list) given prefix[0..n_act]
__device__ __forceinline__ int seg_of(const long long* pre, int n_act, long long g) {
    return upper_bound_ll(pre, n_act + 1, g) - 1;
}
__device__ __forceinline__ int seg_of_int(const int* pre, int n_act, int g) {
    return upper_bound_int(pre, n_act + 1, g) - 1;
}
// seg_of_int for an index g held by every lane of a full warp: each round the
// lanes read 32 evenly spaced entries of the remaining range and vote, so the
// search takes ceil(log32(n_act + 1)) dependent loads instead of log2.
__device__ __forceinline__ int warp_seg_of_int(const int* pre, int n_act, int g) {
    const int lane = threadIdx.x & 31;
    int lo = 0, n = n_act + 1;           // the answer lies in [lo, lo + n), pre[lo] <= g
    for (;;) {
        const int s = (n + 31) >> 5;
        const unsigned v = __ballot_sync(0xffffffffu, lane * s < n && pre[lo + lane * s] <= g);
        const int k = __popc(v) - 1;     // pre is nondecreasing: the true lanes are a prefix
        if (s == 1) return lo + k;
        lo += k * s;
        n = min(s, n - k * s);
    }
}

// A block's copy of a segment prefix table (n_act + 1 entries) in shared
// memory, loaded in one round, so that item -> instance searches do not chain
// dependent global loads; tables longer than SEG_CACHE entries stay global.
// All threads of the block must call it (it synchronises).
constexpr int SEG_CACHE = 512;
template <class PreT>
__device__ __forceinline__ const PreT* seg_table(const PreT* pre, int n_act, PreT* cache) {
    if (n_act + 1 > SEG_CACHE) return pre;
    for (int i = threadIdx.x; i <= n_act; i += blockDim.x) cache[i] = pre[i];
    __syncthreads();
    return cache;
}
// the same with the instance ids of the active list (act) in the same round
template <class PreT>
__device__ __forceinline__ const PreT* seg_table(const PreT* pre, const int* act, int n_act, PreT* cache,
                                                 int* act_cache, const int** act_out) {
    if (n_act + 1 > SEG_CACHE) {
        *act_out = act;
        return pre;
    }
    for (int i = threadIdx.x; i <= n_act; i += blockDim.x) {
        cache[i] = pre[i];
        if (i < n_act) act_cache[i] = act[i];
    }
    __syncthreads();
    *act_out = act_cache;
    return cache;
}

__device__ __forceinline__ unsigned long long hash64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// cheap 32-bit hash of a (lo, hi) key for small shared-memory sets
__device__ __forceinline__ unsigned hash_small(unsigned long long k) {
    return ((unsigned)k * 0x9E3779B1u) ^ ((unsigned)(k >> 32) * 0x85EBCA77u);
}

// Warp-cooperative add of per-lane (key, count) pairs into a shared counted
// set: equal keys are merged across the warp first, then one lane per key
// probes and adds the group's count. Returns false for the lane holding a
// merged group that could not be placed (set full); that lane's `*csum_out`
// carries the group's count.
__device__ __forceinline__ bool warp_set_add(unsigned long long* set, unsigned* cnt, int cap,
                                             unsigned long long key, unsigned c, unsigned* csum_out) {
    const int lane = threadIdx.x & 31;
    const bool has = key != EMPTY_KEY;
    if (!__any_sync(0xffffffffu, has)) return true;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const unsigned csum = __reduce_add_sync(grp, has ? c : 0u);
    *csum_out = csum;
    if (!has || lane != __ffs(grp) - 1) return true;
    unsigned h = hash_small(key) & (cap - 1);
    for (int probe = 0; probe < cap; ++probe) {
        const unsigned long long o = set[h] == key ? key : atomicCAS(&set[h], EMPTY_KEY, key);
        if (o == EMPTY_KEY || o == key) {
            atomicAdd(&cnt[h], csum);
            return true;
        }
        h = (h + 1) & (cap - 1);
    }
    return false;
}

// Warp-aggregated atomic add: lanes that target the same counter are grouped,
// one lane adds the group's sum (far fewer same-address atomics).
__device__ __forceinline__ void warp_add(int* p, int v) {
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, (unsigned long long)p);
    const int sum = __reduce_add_sync(grp, (unsigned)v);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(p, sum);
}

// Warp-aggregated fetch-and-increment: returns a unique old value per lane.
__device__ __forceinline__ int warp_fetch_inc(int* p) {
    const unsigned act = __activemask();
    const unsigned grp = __match_any_sync(act, (unsigned long long)p);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(p, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    return base + __popc(grp & ((1u << lane) - 1u));
}

// Hash tables are allocated for the worst case but used per frame with a
// power-of-two size proportional to the bubble count (small enough to stay in
// L2): returns (2^k - 1) with 2^k >= want, capped by the allocated mask.
__device__ __forceinline__ unsigned dyn_mask(int alloc_mask, long long want) {
    unsigned p = 63u;
    while ((long long)p + 1 < want && p < (unsigned)alloc_mask) p = (p << 1) | 1u;
    return p < (unsigned)alloc_mask ? p : (unsigned)alloc_mask;
}

__device__ __forceinline__ unsigned long long edge_key(int a, int b) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return ((unsigned long long)(unsigned)lo << 32) | (unsigned)hi;
}

// floor division for q > 0
__host__ __device__ inline long long floordiv_ll(long long p, long long q) {
    long long d = p / q;
    if ((p % q != 0) && (p < 0)) d -= 1;
    return d;
}

// insert or add into the (past, now) overlap hash; new keys are listed in olist
__device__ __forceinline__ void ovl_global_insert(const Pools& P, const InstDesc& D, int inst,
                                                  unsigned long long key, unsigned cnt) {
    unsigned long long* H = P.ohash + D.ohash_off;
    unsigned* V = P.oval + D.ohash_off;
    const InstState& S = P.st[inst];
    const unsigned mask = dyn_mask(D.ohash_mask, 8ll * ((long long)S.K + S.K_prev) + 64);
    unsigned h = (unsigned)hash64(key) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = atomicCAS(&H[h], EMPTY_KEY, key);
        if (k == EMPTY_KEY || k == key) {
            atomicAdd(&V[h], cnt);
            if (k == EMPTY_KEY) {
                const int idx = warp_fetch_inc(&P.st[inst].n_ovl);
                if (idx < D.ovl_cap) P.olist[D.ovl_off + idx] = (int)h;
                else if (!(atomicOr(&P.st[inst].err, ERR_OVL_CAP) & (ERR_EDGE_CAP | ERR_OVL_CAP)))
                    atomicAdd(&P.g->lists_over, 1);
            }
            return;
        }
        h = (h + 1) & mask;
    }
    if (!(atomicOr(&P.st[inst].err, ERR_OVL_CAP) & (ERR_EDGE_CAP | ERR_OVL_CAP))) atomicAdd(&P.g->lists_over, 1);
}


// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct Launch {
    long long* nlaunch;  // host counter of kernel launches
    cudaError_t* err;    // first launch error of the step (host)
    bool sequence;       // some instance's past frame is produced in the same step
    bool events;         // some instance classifies its events
    bool centroid_match; // some instance matches by centres
    bool vertex_rule;    // some instance reads its links at Voronoi vertices
    bool masked;         // some instance has walls or obstacles
    cudaStream_t s;
    Pools P;
    StepTable T;
    int grid_items;      // fixed grid for grid-stride item loops
    int total_tilesA, total_tilesV;
    long long total_groups;
    int grid_wide;               // blocks for kernels with one thread per item (pieces, bubbles, links)
    int vpatch;                  // patch layout of the owner kernel (VPATCH_*)
    int graph_inst;              // graph stage with one block per instance (else grid-wide kernels)
};

// patch layouts of the owner kernel (PW x PH sites per patch of a 64 x 32 tile)
enum VPatch : int { VPATCH_8x8 = 0, VPATCH_16x8 = 1, VPATCH_32x8 = 2, VPATCH_16x16 = 3, VPATCH_COUNT = 4 };

// ---------------------------------------------------------------------------
// Checked build (compiled with -DVD_CHECKED into libvd_checked.so): before a
// scatter access whose index is computed from data, vd_in(P, id, i, n) tests
// 0 <= i < n. A failing test records the check's id and the index in
// Globals (the first one of the step is kept), sets ERR_BOUNDS for the step
// (every instance's getters then return VD_ERR_BOUNDS) and returns false, and
// the caller skips the access. The test hook Globals::dbg_chk makes check
// `id` fail without touching memory, to exercise the reporting. In the
// regular build vd_in is the constant true and the checks compile away.
// ---------------------------------------------------------------------------
#ifdef VD_CHECKED
constexpr bool VD_IS_CHECKED = true;
static __device__ __noinline__ bool vd_fail(const Pools& P, int id, long long i) {
    if (atomicCAS(&P.g->chk_id, 0, id) == 0) P.g->chk_index = i;
    atomicOr(&P.g->err, ERR_BOUNDS);
    return false;
}
__device__ __forceinline__ bool vd_in(const Pools& P, int id, long long i, long long n) {
    if (i >= 0 && i < n && *(volatile int*)&P.g->dbg_chk != id) return true;
    return vd_fail(P, id, i);
}
#else
constexpr bool VD_IS_CHECKED = false;
__device__ __forceinline__ bool vd_in(const Pools&, int, long long, long long) { return true; }
#endif

// check ids, one per checked access (reported by vd_debug_check_info)
enum CheckId : int {
    CHK_NONE = 0,
    CHK_TILE_PIECES = 1,     // k_ccl_tiles: piece records of a tile
    CHK_RUN_PIECE = 2,       // k_ccl_tiles: run -> piece table
    CHK_BORDER = 3,          // k_ccl_tiles: border piece ids
    CHK_FGBITS = 4,          // k_ccl_tiles: foreground words
    CHK_MERGE_PARENT = 5,    // k_ccl_merge: piece parents
    CHK_COMP_ID = 6,         // k_comp_accum / k_comp_final: bubble ids
    CHK_WIDE = 7,            // k_comp_accum: wide-piece list
    CHK_BUCKET = 8,          // k_comp_final / k_bucket_scatter: bucket cells and positions
    CHK_RUN_LABEL = 9,       // k_run_labels: run labels
    CHK_OVL_APPEND = 10,     // k_run_labels: appended overlap pairs
    CHK_OWNER = 11,          // k_voronoi: owner writes
    CHK_SCAN_LIST = 12,      // k_voronoi: scanned-centre list
    CHK_KEPT = 13,           // k_voronoi: kept lists
    CHK_LINK_QUEUE = 14,     // k_links: queue of marked sites
    CHK_LINK_LIST = 15,      // k_links / k_links_vertex: per-warp key list
    CHK_EDGE_APPEND = 16,    // appended link keys
    CHK_CSR = 17,            // k_csr_scatter: CSR columns
    CHK_FLIPS = 18,          // k_flip_write: breaking / arising lists
    CHK_SCAN_WRITE = 19,     // k_scan: offsets
    CHK_MATCH = 20,          // k_match_best / k_match_phi: labels of matched pairs
    CHK_COUNT = 21,
};

// Kernels of a step are launched with programmatic dependent launch, so the
// launch of a kernel overlaps the end of the previous one; every step kernel
// begins with pdl_enter(), which waits until the previous kernel has
// completed and its memory is visible. No step kernel touches memory before
// pdl_enter().
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
void launch_step(const Launch& L, void (*kernel)(KArgs...), dim3 grid, dim3 block, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess && L.err && *L.err == cudaSuccess) *L.err = e;
    ++*L.nlaunch;
}


void launch_ccl_tiles(const Launch& L);    // threshold + tile union-find (pass A)
void launch_ccl_rest(const Launch& L);     // border merge, ranks, centroids, bucket grid
void launch_labels(const Launch& L);       // run labels + overlap histogram
void launch_voronoi(const Launch& L);      // exact owner of every site
void launch_links(const Launch& L);        // per-tile links from the owners
void set_kernel_attributes();              // shared-memory carveout of the link kernel
void launch_merge_lists(const Launch& L);  // appended links/pairs -> hash tables
void launch_merge_edges(const Launch& L);     // the links alone (forked step)
void launch_merge_overlaps(const Launch& L);  // the overlap pairs alone (forked step)
void launch_graph_csr_chain(const Launch& L);     // plan + CSR (forked step)
void launch_graph_match_chain(const Launch& L);   // plan + match (forked step)
// graph stage: prefixes of the merged lists, the now-frame CSR, the match,
// the translated past CSR, the flips
void launch_graph_prep(const Launch& L);
void launch_graph_csr(const Launch& L);
void launch_graph_match(const Launch& L);
void launch_graph_flips(const Launch& L);
void launch_graph_inst(const Launch& L);   // the whole graph stage, one block per instance (2 launches)
void launch_begin(const Launch& L);        // per-step counters and field pointers
void launch_finish(const Launch& L);       // swap frames
void launch_edge_keys(cudaStream_t s, const Pools& P, int inst, int slot, unsigned long long* out);
void launch_expand_labels(cudaStream_t s, const Pools& P, int inst, int slot, int* out, int n_tiles);
// every instance's change lists packed at the offsets `off` (3 per instance:
// breaking, arising, active; entry 3n holds the totals)
void launch_gather_changes(cudaStream_t s, const Pools& P, const long long* off, int n, long long nb,
                           unsigned long long* out, unsigned char* act);
// the same for the listed instances only (entry j = instance insts[j])
void launch_gather_changes_list(cudaStream_t s, const Pools& P, const int* insts, const long long* off, int n,
                                long long nb, unsigned long long* out, unsigned char* act);

// generic decoupled look-back scan over a virtual concatenation (vd_scan.cu)
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
enum ScanKind : int {
    SCAN_ROOTBITS = 0,   // popcount of root-bit words
    SCAN_BUCKETS = 1,    // bucket counts
    SCAN_DEG = 2,        // link degrees (now frame)
    SCAN_FLIPS = 3,      // breaking counts per row
    SCAN_FLIPS_A = 4,    // arising counts per row
};
constexpr int SCAN_KINDS = 5;
// the end value of the offset array of scan `kind`, written by k_plan
constexpr int ENDS_NONE = 0;
__host__ __device__ constexpr int ends_bit(ScanKind kind) { return 1 << kind; }
void launch_scan(const Launch& L, ScanKind kind);
void launch_scan2(const Launch& L, ScanKind kind1, ScanKind kind2);   // two scans over the same segments
// recompute prefixes (and bucket grids when with_comp) and the end values of
// the offset arrays whose bits are set in ends; only the prefix arrays whose
// bits are set in pre_mask are written
void launch_plan(const Launch& L, int with_comp, int ends, int pre_mask = PRE_ALL);

}  // namespace vd
