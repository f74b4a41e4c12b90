// Host side of libvd: the C ABI declared in include/vd.h.
//
// A context (vd_ctx) is a batch of one lattice; vd_batch holds many. Both own
// pooled device buffers laid out by instance (InstDesc offsets), a step table
// per active set, and enqueue the same kernel sequence on their stream:
//   begin -> labelling tiles -> border merge -> roots/ranks -> centroids ->
//   bucket grid -> labels + overlap -> Voronoi -> (owner marks) -> links ->
//   CSR of both link directions -> match -> translation + row comparison ->
//   flip lists -> (event classes) -> finish.
// Launches in parentheses run only when some instance of the batch uses the
// option (walls or obstacles, event classes; likewise the centre match and the
// vertex link rule).
// The batch form captures that sequence once into a CUDA graph per active set
// size and replays it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "vd.h"
#include "vd_internal.cuh"

using namespace vd;

namespace {

long long next_pow2(long long v) {
    long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct DevBuf {
    std::vector<void*> ptrs;
    bool ok = true;
    long long bytes = 0;
    template <class T>
    T* alloc(long long n) {
        if (n <= 0) n = 1;
        void* p = nullptr;
        if (cudaMalloc(&p, (size_t)n * sizeof(T)) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        bytes += n * (long long)sizeof(T);
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    void release() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

struct StepTables {
    int n_act = 0;
    int total_tilesA = 0, total_tilesV = 0;
    long long total_groups = 0;
    int* d_act = nullptr;
    int* d_tileA = nullptr;
    int* d_tileV = nullptr;
    long long* d_groups = nullptr;
    long long* d_pre = nullptr;
};

}  // namespace

struct vd_batch {
    int n = 0;
    cudaStream_t s = 0;
    std::vector<InstDesc> desc;
    DevBuf mem;
    Pools P{};
    StepTables all;               // every instance active
    StepTables sub;               // scratch table for subsets
    int grid_items = 0;
    bool any_events = false;           // some instance classifies its events
    bool any_centroid_match = false;   // some instance matches by centres
    bool any_vertex_rule = false;      // some instance reads links at Voronoi vertices
    bool any_masked = false;           // some instance has walls or obstacles
    int vpatch = VPATCH_8x8;           // patch layout of the owner kernel (tuning)
    int graph_inst = 0;                // graph stage with one block per instance (tuning)
    // second stream of a step: the run-label pass, the overlap merge and the
    // match run on it while the owner, link and CSR kernels run on s
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // field pointer tables (device) and their host mirrors
    const float** d_fields = nullptr;
    long long* d_pitches = nullptr;
    std::vector<const float*> h_fields;
    std::vector<long long> h_pitches;
    // host input staging for vd_push_frame_host (instance 0)
    float* d_host_field = nullptr;
    // double-buffered host input (vd_batch_stage_host / vd_batch_push_staged):
    // two sets of input buffers filled on a copy stream
    std::vector<float*> d_stage[2];
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_staged[2] = {nullptr, nullptr};   // copies into buffer k done
    cudaEvent_t ev_read[2] = {nullptr, nullptr};     // the step reading buffer k done
    bool read_pending[2] = {false, false};
    int stage_next = 0;                              // buffer the next stage call fills
    int staged = -1;                                 // staged, not yet pushed
    // graph of the all-active step
    cudaGraphExec_t graph = nullptr;
    bool use_graph = false;
    long long frames_pushed = 0;
    long long launches = 0;
    cudaError_t launch_err = cudaSuccess;   // first failed launch of the step being enqueued
    long long graph_launches = 0;
    bool sequence = false;
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    int ev_used = 0;
    // host copies of the last step's results, filled by the first query after
    // a push: every instance's state in one copy, and every instance's change
    // lists gathered on the device and copied in one piece
    std::vector<InstState> h_st;
    long long st_at = -1;                 // frames_pushed when h_st was filled
    long long chg_at = -1;                // frames_pushed when the lists were filled
    long long chg_nb = 0;                 // breaking entries of all instances
    unsigned long long* d_chg = nullptr;  // [breaking | breaking_prev | arising]
    unsigned long long* h_chg = nullptr;  // pinned
    long long chg_cap = 0;
    unsigned char* d_act = nullptr;       // active flags of all instances
    unsigned char* h_act = nullptr;       // pinned
    long long act_cap = 0;
    // per instance: frames_pushed when its state was last imported (-1: never);
    // until the next push its owners, match and changes are not available
    std::vector<long long> imported_at;
    long long* d_off = nullptr;           // per instance: breaking, arising, active offsets
    long long* h_off = nullptr;           // pinned
};

// default tuning: owner-kernel patches of 8 x 8 sites, buckets of the mean
// centre spacing, a first owner-search round reaching 9 sites beyond the tile
static const int DEFAULT_BUCKET_PCT = 100;
static const int DEFAULT_RING0 = 9;

static const int N_STAGES = 6;
static const char* STAGE_NAMES[N_STAGES] = {
    "labelling tiles (threshold + tile union-find)",
    "bubbles (border merge, ranks, centroids, bucket grid)",
    "run labels + overlap histogram",
    "voronoi owners",
    "links (owner boundaries, plaquettes, merge into hashes)",
    "adjacency, match, translation, flips",
};

struct vd_ctx {
    vd_batch* b;
};

namespace {

vd_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VD_OK : VD_ERR_CUDA; }

bool valid_cfg(const vd_config& c) {
    if (c.Lx < 1 || c.Ly < 1) return false;
    if (c.walls < 0 || c.walls > 3) return false;
    // a bounded axis runs with twice its length
    const long long iLx = (c.walls & 1) ? 2ll * c.Lx : c.Lx, iLy = (c.walls & 2) ? 2ll * c.Ly : c.Ly;
    if (iLx >= (1 << 21) || iLy >= (1 << 21)) return false;   // 1024*L must fit int32
    if (iLx * iLy >= (1ll << 31)) return false;
    if (c.connectivity != 4 && c.connectivity != 8) return false;
    if (c.polarity != VD_ABOVE && c.polarity != VD_BELOW) return false;
    if (c.max_components < 0 || c.max_edges < 0) return false;
    if (c.events != 0 && c.events != 1) return false;
    if (c.match_rule != VD_MATCH_OVERLAP && c.match_rule != VD_MATCH_CENTROID) return false;
    if (c.match_radius < 0) return false;
    if (c.edge_rule != VD_EDGE_ADJ4 && c.edge_rule != VD_EDGE_VERTEX) return false;
    if (c.match_rule == VD_MATCH_CENTROID && (c.match_radius < 1 || c.match_radius > (1 << 20))) return false;
    return true;
}

void build_table(vd_batch* b, const std::vector<int>& act, StepTables& T, bool alloc) {
    const int n = (int)act.size();
    std::vector<int> tA(n + 1, 0), tV(n + 1, 0);
    std::vector<long long> wd(n + 1, 0);
    for (int a = 0; a < n; ++a) {
        const InstDesc& D = b->desc[act[a]];
        tA[a + 1] = tA[a] + D.ntx * D.nty;
        tV[a + 1] = tV[a] + D.vtx * D.vty;
        wd[a + 1] = wd[a] + (long long)D.Ly * D.gpr;
    }
    if (alloc) {
        T.d_act = b->mem.alloc<int>(b->n);
        T.d_tileA = b->mem.alloc<int>(b->n + 1);
        T.d_tileV = b->mem.alloc<int>(b->n + 1);
        T.d_groups = b->mem.alloc<long long>(b->n + 1);
        T.d_pre = b->mem.alloc<long long>((long long)NPRE * (b->n + 1));
        if (!b->mem.ok) return;
    }
    T.n_act = n;
    T.total_tilesA = tA[n];
    T.total_tilesV = tV[n];
    T.total_groups = wd[n];
    cudaMemcpyAsync(T.d_act, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->s);
    cudaMemcpyAsync(T.d_tileA, tA.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->s);
    cudaMemcpyAsync(T.d_tileV, tV.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->s);
    cudaMemcpyAsync(T.d_groups, wd.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, b->s);
}

Launch make_launch(vd_batch* b, const StepTables& T) {
    Launch L;
    L.nlaunch = &b->launches;
    L.err = &b->launch_err;
    L.sequence = b->sequence;
    L.s = b->s;
    L.P = b->P;
    L.T.n_act = T.n_act;
    L.T.act = T.d_act;
    L.T.tileA_pre = T.d_tileA;
    L.T.tileV_pre = T.d_tileV;
    L.T.grp_pre = T.d_groups;
    L.T.pre = T.d_pre;
    L.grid_items = b->grid_items;
    L.events = b->any_events;
    L.centroid_match = b->any_centroid_match;
    L.vertex_rule = b->any_vertex_rule;
    L.masked = b->any_masked;
    L.grid_wide = 4 * b->grid_items;
    L.vpatch = b->vpatch;
    L.graph_inst = b->graph_inst;
    L.total_tilesA = T.total_tilesA;
    L.total_tilesV = T.total_tilesV;
    L.total_groups = T.total_groups;
    return L;
}

cudaEvent_t next_event(vd_batch* b) {
    if (b->ev_used == (int)b->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        b->ev_pool.push_back(e);
    }
    return b->ev_pool[b->ev_used++];
}

void mark(vd_batch* b, bool on) {
    if (!on) return;
    cudaEvent_t e = next_event(b);
    if (e) cudaEventRecord(e, b->s);
}

void note_err(const Launch& L, cudaError_t e) {
    if (e != cudaSuccess && L.err && *L.err == cudaSuccess) *L.err = e;
}

void enqueue_step(vd_batch* b, const Launch& L, bool timed) {
    launch_begin(L);
    mark(b, timed);
    launch_ccl_tiles(L);
    mark(b, timed);
    launch_ccl_rest(L);
    mark(b, timed);
    if (!timed && !L.graph_inst && b->s2) {
        // after the bubble stage two independent chains: run labels ->
        // overlap merge -> match on s2, owners -> links -> link merge -> CSR
        // on s; the flips need both
        Launch L2 = L;
        L2.s = b->s2;
        note_err(L, cudaEventRecord(b->ev_fork, L.s));
        note_err(L, cudaStreamWaitEvent(b->s2, b->ev_fork, 0));
        launch_labels(L2);
        launch_merge_overlaps(L2);
        launch_graph_match_chain(L2);
        note_err(L, cudaEventRecord(b->ev_join, b->s2));
        launch_voronoi(L);
        launch_links(L);
        launch_merge_edges(L);
        launch_graph_csr_chain(L);
        note_err(L, cudaStreamWaitEvent(L.s, b->ev_join, 0));
        launch_graph_flips(L);
        launch_finish(L);
        return;
    }
    launch_labels(L);
    mark(b, timed);
    launch_voronoi(L);
    mark(b, timed);
    launch_links(L);
    launch_merge_lists(L);
    mark(b, timed);
    if (L.graph_inst) {
        launch_graph_inst(L);
    } else {
        launch_graph_prep(L);
        launch_graph_csr(L);
        launch_graph_match(L);
        launch_graph_flips(L);
        launch_finish(L);
    }
    mark(b, timed);
}

vd_status create_batch(const vd_config* cfgs, int n, vd_batch** out, bool sequence = false) {
    if (!cfgs || n < 1 || !out) return VD_ERR_INVALID;
    for (int i = 0; i < n; ++i)
        if (!valid_cfg(cfgs[i])) return VD_ERR_INVALID;
    vd_batch* b = new (std::nothrow) vd_batch();
    if (!b) return VD_ERR_OOM;
    b->n = n;
    b->sequence = sequence && n > 1;
    b->s = (cudaStream_t)cfgs[0].stream;
    b->desc.resize(n);
    long long site = 0, word = 0, grp = 0, tile = 0, border = 0, comp = 0, edge = 0, eh = 0, oh = 0, bucket = 0, ovl = 0;
    long long piece_cap = 0, scan_items = 0, max_sites = 0;
    for (int i = 0; i < n; ++i) {
        const vd_config& c = cfgs[i];
        InstDesc& D = b->desc[i];
        memset(&D, 0, sizeof(D));
        // a bounded axis (walls) runs as a periodic axis of twice the length
        // whose second half is never a bubble
        const int iLx = (c.walls & 1) ? 2 * c.Lx : c.Lx, iLy = (c.walls & 2) ? 2 * c.Ly : c.Ly;
        const long long N = (long long)iLx * iLy, Nu = (long long)c.Lx * c.Ly;
        D.Lx = iLx;
        D.Ly = iLy;
        D.uLx = c.Lx;
        D.uLy = c.Ly;
        D.bucket_pct = DEFAULT_BUCKET_PCT;
        D.ring0 = DEFAULT_RING0;
        D.masked = c.walls ? 1 : 0;
        b->any_masked = b->any_masked || c.walls;
        D.thr = c.threshold;
        D.pol = c.polarity;
        D.events = c.events;
        D.conn8 = c.connectivity == 8 ? 1 : 0;
        D.edge_rule = c.edge_rule;
        b->any_vertex_rule = b->any_vertex_rule || c.edge_rule == VD_EDGE_VERTEX;
        D.match_rule = c.match_rule;
        D.match_radius = c.match_rule == VD_MATCH_CENTROID ? c.match_radius : 0;
        b->any_events = b->any_events || c.events;
        b->any_centroid_match = b->any_centroid_match || c.match_rule == VD_MATCH_CENTROID;
        D.ntx = (iLx + TW - 1) / TW;
        D.nty = (iLy + TH - 1) / TH;
        D.vtx = (iLx + VW - 1) / VW;
        D.vty = (iLy + VH - 1) / VH;
        D.wpr = (iLx + 31) / 32;
        D.gpr = (D.wpr + RGW - 1) / RGW;
        // frame sequence: instance i's past frame is instance i-1 of the same
        // step, instance 0's is instance n-1 of the previous step
        D.seq_prev = sequence ? (i == 0 ? n - 1 : i - 1) : i;
        D.seq_same = (sequence && i > 0) ? 1 : 0;
        long long kcap = c.max_components ? c.max_components
                                          : (Nu <= 65536 ? (Nu + 1) / 2 : std::max<long long>(Nu / 8, 65536));
        kcap = std::min<long long>(kcap, (Nu + 1) / 2);
        long long ecap = c.max_edges ? c.max_edges : 3 * kcap + 64;
        long long ocap = 2 * kcap + 64;
        D.comp_cap = (int)kcap;
        D.edge_cap = (int)ecap;
        D.ovl_cap = (int)ocap;
        D.ehash_mask = (int)(next_pow2(2 * ecap) - 1);
        D.ohash_mask = (int)(next_pow2(2 * ocap) - 1);
        D.bucket_cap = ((iLx + 3) / 4) * ((iLy + 3) / 4);
        D.site_off = site;
        D.word_off = word;
        D.grp_off = grp;
        D.tile_off = tile;
        D.border_off = border;
        D.comp_off = comp;
        D.edge_off = edge;
        D.ehash_off = eh;
        D.ohash_off = oh;
        D.bucket_off = bucket;
        D.ovl_off = ovl;
        const long long ntiles = (long long)D.ntx * D.nty;
        site += N;
        max_sites = std::max(max_sites, N);
        word += (long long)iLy * D.wpr;
        grp += (long long)iLy * D.gpr;
        tile += ntiles;
        border += ntiles * BORDER;
        comp += kcap + 1;
        edge += ecap;
        eh += D.ehash_mask + 1ll;
        oh += D.ohash_mask + 1ll;
        bucket += D.bucket_cap + 1ll;
        ovl += ocap;
        piece_cap += (N <= 65536) ? ntiles * (TSITES / 2) : N / 8 + ntiles * 16;
        scan_items = std::max(scan_items, (long long)0);
    }
    scan_items = std::max(std::max(grp, comp), bucket);
    // the graph stage runs as grid-wide kernels by default: with the step
    // forked into two streams they beat the one-block-per-instance form also
    // for a single 1024^2 lattice; the autotuner tries both
    b->graph_inst = 0;
    if (piece_cap >= (1ll << 31) || comp >= (1ll << 31) || edge >= (1ll << 30)) {
        delete b;
        return VD_ERR_INVALID;
    }
    DevBuf& M = b->mem;
    Pools& P = b->P;
    P.desc = M.alloc<InstDesc>(n);
    P.st = M.alloc<InstState>(n);
    P.g = M.alloc<Globals>(1);
    P.rp = M.alloc<int>(tile * TRUNS);
    P.rl[0] = M.alloc<int>(tile * TRUNS);
    P.rl[1] = M.alloc<int>(tile * TRUNS);
    P.lab_out = M.alloc<int>(max_sites);
    P.owners = M.alloc<int>(site);
    P.fgbits[0] = M.alloc<unsigned>(word);
    P.fgbits[1] = M.alloc<unsigned>(word);
    P.rootbits = M.alloc<unsigned>(word);
    P.obst = M.alloc<unsigned>(word);
    P.rgcnt = M.alloc<int>(grp);
    P.rankpre = M.alloc<int>(grp);
    P.tile_pbase = M.alloc<int>(tile);
    P.tile_pcnt = M.alloc<int>(tile);
    P.border = M.alloc<int>(border);
    P.piece_cap = (int)piece_cap;
    P.p_q = M.alloc<int>(piece_cap);
    P.p_inst = M.alloc<int>(piece_cap);
    P.p_n = M.alloc<int>(piece_cap);
    P.p_su = M.alloc<int>(piece_cap);
    P.p_sv = M.alloc<int>(piece_cap);
    P.p_parent = M.alloc<int>(piece_cap);
    P.p_comp = M.alloc<int>(piece_cap);
    P.p_accn = M.alloc<long long>(piece_cap);
    P.p_accx = M.alloc<long long>(piece_cap);
    P.p_accy = M.alloc<long long>(piece_cap);
    P.wide = M.alloc<int>(piece_cap);
    P.cq[0] = M.alloc<int2>(comp);
    P.cq[1] = M.alloc<int2>(comp);
    P.comp_root = M.alloc<int>(comp);
    P.bcnt = M.alloc<int>(bucket);
    for (int k = 0; k < 2; ++k) {
        P.boff[k] = M.alloc<int>(bucket);
        P.bcq[k] = M.alloc<int2>(comp);
        P.bid[k] = M.alloc<int>(comp);
    }
    P.best_n = M.alloc<unsigned long long>(comp);
    P.best_p = M.alloc<unsigned long long>(comp);
    P.phi = M.alloc<int>(comp);
    P.inv = M.alloc<int>(comp);
    P.active = M.alloc<unsigned char>(comp);
    P.deg = M.alloc<int>(comp);
    P.rowoff[0] = M.alloc<int>(comp);
    P.rowoff[1] = M.alloc<int>(comp);
    P.tlen = M.alloc<int>(comp);
    P.fcnt = M.alloc<int>(comp);
    P.fcnt_a = M.alloc<int>(comp);
    P.foff = M.alloc<int>(comp);
    P.foff_a = M.alloc<int>(comp);
    P.cols[0] = M.alloc<int>(2 * edge);
    P.cols[1] = M.alloc<int>(2 * edge);
    P.tcols = M.alloc<int>(2 * edge);
    P.ehash = M.alloc<unsigned long long>(eh);
    P.elist = M.alloc<int>(edge);
    P.ohash = M.alloc<unsigned long long>(oh);
    P.oval = M.alloc<unsigned>(oh);
    P.olist = M.alloc<int>(ovl);
    P.brk = M.alloc<unsigned long long>(edge);
    P.brk_prev = M.alloc<unsigned long long>(edge);
    P.ari = M.alloc<unsigned long long>(edge);
    P.ekeys = M.alloc<unsigned long long>(edge);
    P.oapp_key = M.alloc<unsigned long long>(ovl);
    P.oapp_cnt = M.alloc<unsigned>(ovl);
    P.scan_flag_cap = scan_items / SCAN_TILE + 2;
    P.scan_flags = M.alloc<unsigned long long>(SCAN_KINDS * P.scan_flag_cap);
    b->d_fields = M.alloc<const float*>(n);
    b->d_pitches = M.alloc<long long>(n);
    P.fields = b->d_fields;
    P.pitches = b->d_pitches;
    if (!M.ok) {
        M.release();
        delete b;
        return VD_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaMemcpyAsync(P.desc, b->desc.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, b->s));
    chk(cudaMemsetAsync(P.st, 0, sizeof(InstState) * n, b->s));
    chk(cudaMemsetAsync(P.g, 0, sizeof(Globals), b->s));
    chk(cudaMemsetAsync(P.rl[0], 0xff, sizeof(int) * tile * TRUNS, b->s));
    chk(cudaMemsetAsync(P.rl[1], 0xff, sizeof(int) * tile * TRUNS, b->s));
    chk(cudaMemsetAsync(P.rootbits, 0, sizeof(unsigned) * word, b->s));
    chk(cudaMemsetAsync(P.obst, 0, sizeof(unsigned) * word, b->s));
    chk(cudaMemsetAsync(P.rgcnt, 0, sizeof(int) * grp, b->s));
    chk(cudaMemsetAsync(P.bcnt, 0, sizeof(int) * bucket, b->s));
    chk(cudaMemsetAsync(P.deg, 0, sizeof(int) * comp, b->s));
    chk(cudaMemsetAsync(P.best_n, 0, sizeof(unsigned long long) * comp, b->s));
    chk(cudaMemsetAsync(P.rowoff[0], 0, sizeof(int) * comp, b->s));
    chk(cudaMemsetAsync(P.rowoff[1], 0, sizeof(int) * comp, b->s));
    chk(cudaMemsetAsync(P.ehash, 0xff, sizeof(unsigned long long) * eh, b->s));
    chk(cudaMemsetAsync(P.ohash, 0xff, sizeof(unsigned long long) * oh, b->s));
    chk(cudaMemsetAsync(P.oval, 0, sizeof(unsigned) * oh, b->s));
    chk(cudaMemsetAsync(P.scan_flags, 0, sizeof(unsigned long long) * SCAN_KINDS * P.scan_flag_cap, b->s));
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid_items = 2 * sms;
    set_kernel_attributes();
    if (cudaStreamCreateWithFlags(&b->s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        M.ok = false;
    }
    std::vector<int> act(n);
    for (int i = 0; i < n; ++i) act[i] = i;
    build_table(b, act, b->all, true);
    build_table(b, act, b->sub, true);
    b->h_fields.assign(n, nullptr);
    b->h_pitches.assign(n, 0);
    b->imported_at.assign(n, -1);

    if (!M.ok) {
        if (b->s2) cudaStreamDestroy(b->s2);
        if (b->ev_fork) cudaEventDestroy(b->ev_fork);
        if (b->ev_join) cudaEventDestroy(b->ev_join);
        M.release();
        delete b;
        return VD_ERR_OOM;
    }
    chk(cudaStreamSynchronize(b->s));
    if (e != cudaSuccess) {
        cudaStreamDestroy(b->s2);
        cudaEventDestroy(b->ev_fork);
        cudaEventDestroy(b->ev_join);
        M.release();
        delete b;
        return VD_ERR_CUDA;
    }
    *out = b;
    return VD_OK;
}

// state of instance i after the last push; the first call after a push waits
// for the stream and copies every instance's state at once
vd_status read_state(vd_batch* b, int i, InstState* st) {
    if (!b || i < 0 || i >= b->n) return VD_ERR_INVALID;
    if (b->st_at != b->frames_pushed) {
        cudaError_t e = cudaStreamSynchronize(b->s);
        if (e != cudaSuccess) return VD_ERR_CUDA;
        b->h_st.resize(b->n);
        e = cudaMemcpy(b->h_st.data(), b->P.st, sizeof(InstState) * b->n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return VD_ERR_CUDA;
        b->st_at = b->frames_pushed;
    }
    *st = b->h_st[i];
    return VD_OK;
}

// change lists of every instance of the last push in host memory: offsets
// from the cached states, one gather kernel into a packed device buffer, one
// copy to pinned host memory
vd_status ensure_changes(vd_batch* b) {
    if (b->chg_at == b->frames_pushed) return VD_OK;
    InstState tmp;
    vd_status r = read_state(b, 0, &tmp);
    if (r) return r;
    const int n = b->n;
    if (!b->h_off) {
        if (cudaMallocHost(&b->h_off, sizeof(long long) * 3 * (n + 1)) != cudaSuccess) return VD_ERR_OOM;
        if (cudaMalloc(&b->d_off, sizeof(long long) * 3 * (n + 1)) != cudaSuccess) return VD_ERR_OOM;
    }
    long long nb = 0, na = 0, nk = 0;
    for (int j = 0; j < n; ++j) {
        const InstState& s = b->h_st[j];
        b->h_off[3 * j] = nb;
        b->h_off[3 * j + 1] = na;
        b->h_off[3 * j + 2] = nk;
        if (s.frame > 0 && !s.err) {
            nb += s.n_break;
            na += s.n_arise;
            nk += s.K;
        }
    }
    b->h_off[3 * n] = nb;
    b->h_off[3 * n + 1] = na;
    b->h_off[3 * n + 2] = nk;
    const long long need = 2 * nb + na;
    if (need > b->chg_cap) {
        cudaFree(b->d_chg);
        cudaFreeHost(b->h_chg);
        b->d_chg = nullptr;
        b->h_chg = nullptr;
        b->chg_cap = 0;
        const long long cap = need + need / 2 + 1024;
        if (cudaMalloc(&b->d_chg, sizeof(unsigned long long) * cap) != cudaSuccess) return VD_ERR_OOM;
        if (cudaMallocHost(&b->h_chg, sizeof(unsigned long long) * cap) != cudaSuccess) return VD_ERR_OOM;
        b->chg_cap = cap;
    }
    if (nk > b->act_cap) {
        cudaFree(b->d_act);
        cudaFreeHost(b->h_act);
        b->d_act = nullptr;
        b->h_act = nullptr;
        b->act_cap = 0;
        const long long cap = nk + nk / 2 + 1024;
        if (cudaMalloc(&b->d_act, cap) != cudaSuccess) return VD_ERR_OOM;
        if (cudaMallocHost(&b->h_act, cap) != cudaSuccess) return VD_ERR_OOM;
        b->act_cap = cap;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_off, b->h_off, sizeof(long long) * 3 * (n + 1), cudaMemcpyHostToDevice, b->s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
    launch_gather_changes(b->s, b->P, b->d_off, n, nb, b->d_chg, b->d_act);
    b->launches += 1;
    if (need > 0) e = cudaMemcpyAsync(b->h_chg, b->d_chg, sizeof(unsigned long long) * need, cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess && nk > 0) e = cudaMemcpyAsync(b->h_act, b->d_act, nk, cudaMemcpyDeviceToHost, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
    b->chg_nb = nb;
    b->chg_at = b->frames_pushed;
    return VD_OK;
}

// copy from host staging into a caller buffer in host or device memory
vd_status copy_from_host(void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return VD_OK;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, dst) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return cuda_status(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
    std::memcpy(dst, src, bytes);
    return VD_OK;
}

vd_status err_status(const InstState& st) {
    if (st.err & ERR_BOUNDS) return VD_ERR_BOUNDS;
    if (st.err & ERR_TIMEOUT) return VD_ERR_TIMEOUT;
    if (st.err) return VD_ERR_CAPACITY;
    return VD_OK;
}

vd_status push_fields(vd_batch* b, const std::vector<int>& act, const float* const* fields, const long long* pitches) {
    for (size_t a = 0; a < act.size(); ++a) {
        if (!fields[a]) return VD_ERR_INVALID;
        b->h_fields[act[a]] = fields[a];
        b->h_pitches[act[a]] = pitches[a];
    }
    // small copies from pageable memory: the runtime stages them before it
    // returns (the vectors may change right after) and they do not queue on a
    // copy engine behind a large staged frame copy, as pinned copies would
    cudaError_t e = cudaMemcpyAsync(b->d_fields, b->h_fields.data(), sizeof(float*) * b->n, cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_pitches, b->h_pitches.data(), sizeof(long long) * b->n, cudaMemcpyHostToDevice, b->s);
    return cuda_status(e);
}

// status of the step just enqueued: a failed launch, else the runtime's
// last error
vd_status step_status(vd_batch* b) {
    const cudaError_t le = b->launch_err;
    b->launch_err = cudaSuccess;
    const cudaError_t e = cudaGetLastError();
    return cuda_status(le != cudaSuccess ? le : e);
}

vd_status run_all(vd_batch* b) {
    const Launch L = make_launch(b, b->all);
    b->frames_pushed += 1;
    if (b->timing) {
        enqueue_step(b, L, true);
        return step_status(b);
    }
    if (b->use_graph) {
        if (!b->graph) {
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return VD_ERR_CUDA;
            const long long before = b->launches;
            enqueue_step(b, L, false);
            b->graph_launches = b->launches - before;
            b->launches = before;
            e = cudaStreamEndCapture(b->s, &g);
            if (e != cudaSuccess) return VD_ERR_CUDA;
            if (step_status(b)) {
                cudaGraphDestroy(g);
                return VD_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return VD_ERR_CUDA;
        }
        b->launches += b->graph_launches;
        return cuda_status(cudaGraphLaunch(b->graph, b->s));
    }
    enqueue_step(b, L, false);
    return step_status(b);
}

vd_status copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return VD_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

// the state of instance i was imported and no frame has been pushed since:
// the imported state holds no owners, match or changes
bool fresh_import(const vd_batch* b, int i) { return b->imported_at[i] == b->frames_pushed; }

vd_status get_changes(vd_batch* b, int i, vd_changes* out) {
    if (!out) return VD_ERR_INVALID;
    InstState st;
    vd_status rs = read_state(b, i, &st);
    if (rs) return rs;
    if (st.frame == 0 || fresh_import(b, i)) return VD_ERR_STATE;
    const InstDesc& D = b->desc[i];
    out->frame_index = b->sequence ? (st.frame - 1) * b->n + i : st.frame - 1;
    out->n_prev = st.rep_K_prev;
    out->n_now = st.K;
    out->n_matched = st.n_matched;
    out->n_edges = st.E;
    out->n_breaking = st.n_break;
    out->n_arising = st.n_arise;
    out->global_trigger = (st.n_break + st.n_arise) > 0;
    vd_status es = err_status(st);
    if (es) return es;
    bool fit = true;
    if (st.n_break > 0 && (!out->breaking || out->cap_breaking < st.n_break)) fit = false;
    if (st.n_arise > 0 && (!out->arising || out->cap_arising < st.n_arise)) fit = false;
    if (out->active && out->cap_active < st.K) fit = false;
    if (!fit) return VD_ERR_CAPACITY;
    vd_status r = ensure_changes(b);
    if (r) return r;
    const size_t u8 = sizeof(unsigned long long);
    const long long ob = b->h_off[3 * i], oa = b->h_off[3 * i + 1], ok = b->h_off[3 * i + 2];
    if (st.n_break > 0) {
        r = copy_from_host(out->breaking, b->h_chg + ob, u8 * st.n_break);
        if (!r && out->breaking_prev) r = copy_from_host(out->breaking_prev, b->h_chg + b->chg_nb + ob, u8 * st.n_break);
    }
    if (!r && st.n_arise > 0) r = copy_from_host(out->arising, b->h_chg + 2 * b->chg_nb + oa, u8 * st.n_arise);
    if (!r && out->active && st.K > 0) r = copy_from_host(out->active, b->h_act + ok, st.K);
    (void)D;
    return r;
}

vd_status get_array(vd_batch* b, int i, int which, void* out, int64_t cap, int64_t* n) {
    if (!out && cap > 0) return VD_ERR_INVALID;
    InstState st;
    vd_status rs = read_state(b, i, &st);
    if (rs) return rs;
    if (st.frame == 0) return VD_ERR_STATE;
    if (fresh_import(b, i) && (which == 1 || which == 4 || which == 5)) return VD_ERR_STATE;
    const InstDesc& D = b->desc[i];
    const long long N = (long long)D.Lx * D.Ly;
    const int slot = st.slot;   // the frame just finished
    long long cnt = 0;
    size_t esz = 4;
    switch (which) {
        case 0: case 1: cnt = (long long)D.uLx * D.uLy; break;
        case 2: cnt = 2ll * st.K; break;
        case 3: cnt = st.E; esz = 8; break;
        case 4: cnt = st.rep_K_prev; break;
        case 5: cnt = st.K; esz = 1; break;
        default: return VD_ERR_INVALID;
    }
    if (n) *n = cnt;
    // a failed frame's state is not read by any kernel
    vd_status es = err_status(st);
    if (es) return es;
    if (cap < cnt) return VD_ERR_CAPACITY;
    const void* src = nullptr;
    switch (which) {
        case 0:
            launch_expand_labels(b->s, b->P, i, slot, b->P.lab_out, D.ntx * D.nty);
            src = b->P.lab_out;
            break;
        case 1: src = b->P.owners + D.site_off; break;
        case 2: src = b->P.cq[slot] + D.comp_off; break;
        case 3:
            launch_edge_keys(b->s, b->P, i, slot, b->P.ekeys + D.edge_off);
            src = b->P.ekeys + D.edge_off;
            break;
        case 4: src = b->P.phi + D.comp_off; break;
        default: src = b->P.active + D.comp_off; break;
    }
    if ((which == 0 || which == 1) && (D.uLx != D.Lx || D.uLy != D.Ly)) {
        // a bounded axis runs with twice its length: return the domain only
        if (cnt == 0) return VD_OK;
        cudaError_t e = cudaMemcpy2DAsync(out, sizeof(int) * D.uLx, src, sizeof(int) * D.Lx, sizeof(int) * D.uLx,
                                          D.uLy, cudaMemcpyDefault, b->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
        return cuda_status(e);
    }
    return copy_out(out, src, (size_t)cnt * esz, b->s);
}

// ---------------------------------------------------------------------------
// Checkpoint / resume of one instance (vd_export_state / vd_import_state).
// The state a frame leaves for the next one (Section 3.2.3 compares each frame
// with the previous one): its foreground bits and run labels (the labels),
// its centroids and their bucket grid, and its links as a CSR of both
// directions, plus the frame count. Blob = StateHeader + those arrays in that
// order, native byte order; the header carries the lattice, the counts and an
// FNV-1a checksum of the arrays, and import checks every value's range, so a
// damaged or foreign blob is refused before anything reaches the device.
// ---------------------------------------------------------------------------
constexpr uint32_t STATE_MAGIC = 0x31534456u;   // "VDS1"
constexpr uint32_t STATE_VERSION = 2;   // 2: run tables packed per tile (row-major run order)

struct StateHeader {
    uint32_t magic, version;
    int32_t Lx, Ly, uLx, uLy;   // lattice as run (a bounded axis runs with twice its length) and as seen
    int32_t K, E;               // bubbles and links of the frame
    int32_t B, nbx, nby, pad;   // its bucket grid
    int64_t frame;              // frames finished
    int64_t n_words, n_runs;    // foreground words, run-label slots
    uint64_t checksum;          // FNV-1a 64 of the arrays
};

struct StateLayout {
    long long words, runs, K, nb, E;
    size_t o_fg, o_rl, o_cq, o_boff, o_bcq, o_bid, o_ro, o_cols, total;
};

StateLayout state_layout(const InstDesc& D, int K, int E, int nb) {
    StateLayout L;
    L.words = (long long)D.Ly * D.wpr;
    L.runs = (long long)D.ntx * D.nty * TRUNS;
    L.K = K;
    L.nb = nb;
    L.E = E;
    size_t o = sizeof(StateHeader);
    L.o_fg = o; o += sizeof(unsigned) * L.words;
    L.o_rl = o; o += sizeof(int) * L.runs;
    L.o_cq = o; o += sizeof(int2) * K;
    L.o_boff = o; o += sizeof(int) * (nb + 1);
    L.o_bcq = o; o += sizeof(int2) * K;
    L.o_bid = o; o += sizeof(int) * K;
    L.o_ro = o; o += sizeof(int) * (K + 1);
    L.o_cols = o; o += sizeof(int) * 2ll * E;
    L.total = o;
    return L;
}

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t k = 0; k < n; ++k) {
        h ^= p[k];
        h *= 1099511628211ull;
    }
    return h;
}

vd_status export_state(vd_batch* b, int i, void* buf, int64_t cap, int64_t* n_bytes) {
    if (!b || i < 0 || i >= b->n) return VD_ERR_INVALID;
    if (b->sequence) return VD_ERR_UNSUPPORTED;   // a sequence's frames are not independent lattices
    InstState st;
    vd_status r = read_state(b, i, &st);
    if (r) return r;
    if (st.frame == 0) return VD_ERR_STATE;
    r = err_status(st);
    if (r) return r;
    const InstDesc& D = b->desc[i];
    const int slot = st.slot;
    const int K = st.Kb[slot], E = st.Eb[slot];
    const int nb = K > 0 ? st.nbxs[slot] * st.nbys[slot] : 0;
    const StateLayout L = state_layout(D, K, E, nb);
    if (n_bytes) *n_bytes = (int64_t)L.total;
    if (!buf || cap < (int64_t)L.total) return VD_ERR_CAPACITY;
    unsigned char* o = static_cast<unsigned char*>(buf);
    const Pools& P = b->P;
    cudaError_t e = cudaSuccess;
    auto get = [&](size_t off, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(o + off, src, bytes, cudaMemcpyDeviceToHost, b->s);
    };
    get(L.o_fg, P.fgbits[slot] + D.word_off, sizeof(unsigned) * L.words);
    get(L.o_rl, P.rl[slot] + D.tile_off * TRUNS, sizeof(int) * L.runs);
    get(L.o_cq, P.cq[slot] + D.comp_off, sizeof(int2) * K);
    get(L.o_boff, P.boff[slot] + D.bucket_off, sizeof(int) * (nb + 1));
    get(L.o_bcq, P.bcq[slot] + D.comp_off, sizeof(int2) * K);
    get(L.o_bid, P.bid[slot] + D.comp_off, sizeof(int) * K);
    get(L.o_ro, P.rowoff[slot] + D.comp_off, sizeof(int) * (K + 1));
    get(L.o_cols, P.cols[slot] + 2 * D.edge_off, sizeof(int) * 2ll * E);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
    if (K == 0) {   // the grid of an empty frame is never read; store its end offset as 0
        int z = 0;
        std::memcpy(o + L.o_boff, &z, sizeof(int));
    }
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = STATE_MAGIC;
    h.version = STATE_VERSION;
    h.Lx = D.Lx;
    h.Ly = D.Ly;
    h.uLx = D.uLx;
    h.uLy = D.uLy;
    h.K = K;
    h.E = E;
    h.B = st.Bs[slot];
    h.nbx = K > 0 ? st.nbxs[slot] : 0;
    h.nby = K > 0 ? st.nbys[slot] : 0;
    h.frame = st.frame;
    h.n_words = L.words;
    h.n_runs = L.runs;
    h.checksum = fnv1a(o + sizeof(StateHeader), L.total - sizeof(StateHeader));
    std::memcpy(o, &h, sizeof(h));
    return VD_OK;
}

// every value of a blob in the range the kernels assume
bool state_values_ok(const InstDesc& D, const StateHeader& h, const StateLayout& L, const unsigned char* o) {
    const int K = h.K, E = h.E;
    auto at = [&](size_t off, long long k) {
        int v;
        std::memcpy(&v, o + off + sizeof(int) * k, sizeof(int));
        return v;
    };
    // foreground bits only inside the lattice (and its first half on a bounded axis)
    for (int y = 0; y < D.Ly; ++y)
        for (int w = 0; w < D.wpr; ++w) {
            unsigned v;
            std::memcpy(&v, o + L.o_fg + sizeof(unsigned) * ((long long)y * D.wpr + w), sizeof(unsigned));
            const int x0 = 32 * w;
            const int lim = y < D.uLy ? std::min(D.uLx, D.Lx) : 0;
            const unsigned allowed = x0 >= lim ? 0u : (lim - x0 >= 32 ? ~0u : ((1u << (lim - x0)) - 1u));
            if (v & ~allowed) return false;
        }
    for (long long k = 0; k < L.runs; ++k) {
        const int v = at(L.o_rl, k);
        if (v < -1 || v >= K) return false;
    }
    const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
    for (long long k = 0; k < 2ll * K; ++k) {
        const long long v = at(L.o_cq, k), M = (k & 1) ? MY : MX;
        if (v < 0 || v >= M) return false;
    }
    int prev = 0;
    for (long long k = 0; k <= L.nb; ++k) {
        const int v = at(L.o_boff, k);
        if (v < prev || v > K) return false;
        prev = v;
    }
    if (at(L.o_boff, L.nb) != (L.nb > 0 ? K : 0)) return false;
    // bucket order: entry j of bucket k is centre bid[j], stored in that bucket
    for (long long k = 0; k < L.nb; ++k)
        for (int j = at(L.o_boff, k); j < at(L.o_boff, k + 1); ++j) {
            const int id = at(L.o_bid, j);
            if (id < 0 || id >= K) return false;
            const int bx = at(L.o_bcq, 2ll * j), by = at(L.o_bcq, 2ll * j + 1);
            if (bx != at(L.o_cq, 2ll * id) || by != at(L.o_cq, 2ll * id + 1)) return false;
            if ((long long)(by / Q / h.B) * h.nbx + (bx / Q / h.B) != k) return false;
        }
    // CSR rows: ascending labels, no self link
    prev = 0;
    for (long long k = 0; k <= K; ++k) {
        const int v = at(L.o_ro, k);
        if (v < prev || v > 2 * E) return false;
        prev = v;
    }
    if (at(L.o_ro, K) != 2 * E) return false;
    for (long long a = 0; a < K; ++a)
        for (int j = at(L.o_ro, a); j < at(L.o_ro, a + 1); ++j) {
            const int v = at(L.o_cols, j);
            if (v < 0 || v >= K || v == a) return false;
            if (j > at(L.o_ro, a) && v <= at(L.o_cols, j - 1)) return false;
        }
    return true;
}

vd_status import_state(vd_batch* b, int i, const void* buf, int64_t n_bytes) {
    if (!b || i < 0 || i >= b->n || !buf) return VD_ERR_INVALID;
    if (b->sequence) return VD_ERR_UNSUPPORTED;
    if (n_bytes < (int64_t)sizeof(StateHeader)) return VD_ERR_INVALID;
    const unsigned char* o = static_cast<const unsigned char*>(buf);
    StateHeader h;
    std::memcpy(&h, o, sizeof(h));
    const InstDesc& D = b->desc[i];
    if (h.magic != STATE_MAGIC || h.version != STATE_VERSION) return VD_ERR_INVALID;
    if (h.Lx != D.Lx || h.Ly != D.Ly || h.uLx != D.uLx || h.uLy != D.uLy) return VD_ERR_INVALID;
    if (h.frame < 1 || h.K < 0 || h.E < 0 || h.K > D.comp_cap || h.E > D.edge_cap) return VD_ERR_INVALID;
    if (h.K > 0 && (h.B < 4 || h.B > 64 || h.nbx != (D.Lx + h.B - 1) / h.B || h.nby != (D.Ly + h.B - 1) / h.B))
        return VD_ERR_INVALID;
    if (h.K == 0 && (h.nbx != 0 || h.nby != 0)) return VD_ERR_INVALID;
    const int nb = h.K > 0 ? h.nbx * h.nby : 0;
    if (nb > D.bucket_cap) return VD_ERR_INVALID;
    const StateLayout L = state_layout(D, h.K, h.E, nb);
    if (h.n_words != L.words || h.n_runs != L.runs || n_bytes != (int64_t)L.total) return VD_ERR_INVALID;
    if (fnv1a(o + sizeof(StateHeader), L.total - sizeof(StateHeader)) != h.checksum) return VD_ERR_INVALID;
    if (!state_values_ok(D, h, L, o)) return VD_ERR_INVALID;
    InstState st;
    vd_status r = read_state(b, i, &st);   // waits for the stream
    if (r) return r;
    const int slot = st.slot;
    const Pools& P = b->P;
    cudaError_t e = cudaSuccess;
    auto put = [&](void* dst, size_t off, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, o + off, bytes, cudaMemcpyHostToDevice, b->s);
    };
    put(P.fgbits[slot] + D.word_off, L.o_fg, sizeof(unsigned) * L.words);
    put(P.rl[slot] + D.tile_off * TRUNS, L.o_rl, sizeof(int) * L.runs);
    put(P.cq[slot] + D.comp_off, L.o_cq, sizeof(int2) * h.K);
    put(P.boff[slot] + D.bucket_off, L.o_boff, sizeof(int) * (nb + 1));
    put(P.bcq[slot] + D.comp_off, L.o_bcq, sizeof(int2) * h.K);
    put(P.bid[slot] + D.comp_off, L.o_bid, sizeof(int) * h.K);
    put(P.rowoff[slot] + D.comp_off, L.o_ro, sizeof(int) * (h.K + 1));
    put(P.cols[slot] + 2 * D.edge_off, L.o_cols, sizeof(int) * 2ll * h.E);
    // the instance's state: the imported frame is its last finished frame
    st.Kb[slot] = h.K;
    st.Eb[slot] = h.E;
    st.Bs[slot] = h.K > 0 ? h.B : 4;
    st.nbxs[slot] = h.nbx;
    st.nbys[slot] = h.nby;
    st.B = st.Bs[slot];
    st.nbx = h.nbx;
    st.nby = h.nby;
    st.frame = h.frame;
    st.last_ok = 1;
    st.K = h.K;
    st.E = h.E;
    st.E_prev = h.E;
    st.K_prev = 0;
    st.rep_K_prev = 0;
    st.K_roots = h.K;
    st.n_matched = 0;
    st.n_break = 0;
    st.n_arise = 0;
    if (st.err & (ERR_EDGE_CAP | ERR_OVL_CAP)) {
        // the instance's last frame overflowed a list: its hash tables keep
        // unlisted keys that its next step would have cleared; clear them here
        // and take it off the count of such instances
        const InstDesc& Di = b->desc[i];
        if (e == cudaSuccess && (st.err & ERR_EDGE_CAP))
            e = cudaMemsetAsync(P.ehash + Di.ehash_off, 0xff, sizeof(unsigned long long) * (Di.ehash_mask + 1ll), b->s);
        if (e == cudaSuccess && (st.err & ERR_OVL_CAP))
            e = cudaMemsetAsync(P.ohash + Di.ohash_off, 0xff, sizeof(unsigned long long) * (Di.ohash_mask + 1ll), b->s);
        if (e == cudaSuccess && (st.err & ERR_OVL_CAP))
            e = cudaMemsetAsync(P.oval + Di.ohash_off, 0, sizeof(unsigned) * (Di.ohash_mask + 1ll), b->s);
        int over = 0;
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
        if (e == cudaSuccess) e = cudaMemcpy(&over, &P.g->lists_over, sizeof(int), cudaMemcpyDeviceToHost);
        over = over > 0 ? over - 1 : 0;
        if (e == cudaSuccess) e = cudaMemcpy(&P.g->lists_over, &over, sizeof(int), cudaMemcpyHostToDevice);
    }
    st.err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.st + i, &st, sizeof(InstState), cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
    b->st_at = -1;
    b->chg_at = -1;
    b->imported_at[i] = b->frames_pushed;
    return VD_OK;
}

// obstacle bits of instance i from a host byte mask (uLy rows of `pitch` bytes)
vd_status set_obstacles(vd_batch* b, int i, const uint8_t* h_mask, int64_t pitch) {
    if (!b || i < 0 || i >= b->n || !h_mask) return VD_ERR_INVALID;
    InstDesc& D = b->desc[i];
    if (pitch < D.uLx) return VD_ERR_INVALID;
    std::vector<unsigned> bits((size_t)D.Ly * D.wpr, 0u);
    bool any = false;
    for (int y = 0; y < D.uLy; ++y)
        for (int x = 0; x < D.uLx; ++x)
            if (h_mask[(long long)y * pitch + x]) {
                bits[(size_t)y * D.wpr + (x >> 5)] |= 1u << (x & 31);
                any = true;
            }
    cudaError_t e = cudaMemcpyAsync(b->P.obst + D.word_off, bits.data(), sizeof(unsigned) * bits.size(),
                                    cudaMemcpyHostToDevice, b->s);
    const int masked = (D.uLx != D.Lx || D.uLy != D.Ly || any) ? 1 : 0;
    if (e == cudaSuccess && masked != D.masked) {
        D.masked = masked;
        e = cudaMemcpyAsync(b->P.desc + i, &D, sizeof(InstDesc), cudaMemcpyHostToDevice, b->s);
        if (masked && !b->any_masked) {
            // the step gains the owner-marking launch: capture the graph again
            b->any_masked = true;
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);   // `bits` is released on return
    return cuda_status(e);
}

}  // namespace

namespace vd {
// per-step results of some instances, gathered on the device and copied
// asynchronously into pinned host memory: 8 ints per instance
// (K, E, n_breaking, n_arising, n_matched, err, past-frame bubbles, frames finished)
__global__ void k_gather_counts(Pools P, const int* sims, int n, int* out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const InstState& S = P.st[sims[k]];
        out[8 * k + 0] = S.K;
        out[8 * k + 1] = S.E;
        out[8 * k + 2] = S.n_break;
        out[8 * k + 3] = S.n_arise;
        out[8 * k + 4] = S.n_matched;
        out[8 * k + 5] = S.err;
        out[8 * k + 6] = S.rep_K_prev;
        out[8 * k + 7] = (int)S.frame;
    }
}
}  // namespace vd

long long vd_batch_resident_bytes(const vd_batch* b) { return b ? b->mem.bytes : 0; }

vd_status vd_batch_gather_counts_async(vd_batch* b, const int* h_sims, int n, int* d_scratch, int* h_pinned_out) {
    if (!b || n <= 0) return VD_ERR_INVALID;
    int* d_sims = d_scratch;
    int* d_out = d_scratch + n;   // 8 ints per instance follow the n instance ids
    if (cudaMemcpyAsync(d_sims, h_sims, sizeof(int) * n, cudaMemcpyHostToDevice, b->s) != cudaSuccess) return VD_ERR_CUDA;
    vd::k_gather_counts<<<1, 256, 0, b->s>>>(b->P, d_sims, n, d_out);
    b->launches += 1;
    if (cudaMemcpyAsync(h_pinned_out, d_out, sizeof(int) * 8 * n, cudaMemcpyDeviceToHost, b->s) != cudaSuccess)
        return VD_ERR_CUDA;
    return VD_OK;
}

// change lists of the listed instances packed into d_out / d_act on `stream`
// (see launch_gather_changes_list); the caller orders it after their step
vd_status vd_batch_gather_changes_list_async(vd_batch* b, void* stream, const int* d_insts, const long long* d_off,
                                             int n, long long nb, uint64_t* d_out, uint8_t* d_act) {
    if (!b || n <= 0) return VD_ERR_INVALID;
    launch_gather_changes_list((cudaStream_t)stream, b->P, d_insts, d_off, n, nb,
                               reinterpret_cast<unsigned long long*>(d_out), d_act);
    b->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? VD_OK : VD_ERR_CUDA;
}

extern "C" {

vd_status vd_config_init(vd_config* cfg, int32_t Lx, int32_t Ly) {
    if (!cfg) return VD_ERR_INVALID;
    memset(cfg, 0, sizeof(*cfg));
    cfg->Lx = Lx;
    cfg->Ly = Ly;
    cfg->threshold = 0.5f;
    cfg->polarity = VD_ABOVE;
    cfg->connectivity = 4;
    return VD_OK;
}

const char* vd_status_string(vd_status s) {
    switch (s) {
        case VD_OK: return "ok";
        case VD_ERR_INVALID: return "invalid argument";
        case VD_ERR_OOM: return "device allocation failed";
        case VD_ERR_CAPACITY: return "capacity exceeded";
        case VD_ERR_CUDA: return "CUDA runtime error";
        case VD_ERR_TIMEOUT: return "bounded device wait expired";
        case VD_ERR_STATE: return "call out of order";
        case VD_ERR_UNSUPPORTED: return "unsupported";
        case VD_ERR_BOUNDS: return "an index check of the checked build failed";
        default: return "unknown status";
    }
}

vd_status vd_create(const vd_config* cfg, vd_ctx** out) {
    if (!cfg || !out) return VD_ERR_INVALID;
    vd_batch* b = nullptr;
    vd_status r = create_batch(cfg, 1, &b);
    if (r) return r;
    // graph replay needs a capturable stream (not the legacy default stream)
    b->use_graph = (cfg->stream != nullptr);
    vd_ctx* c = new (std::nothrow) vd_ctx();
    if (!c) {
        b->mem.release();
        delete b;
        return VD_ERR_OOM;
    }
    c->b = b;
    *out = c;
    return VD_OK;
}

vd_status vd_push_frame(vd_ctx* ctx, const float* d_field, size_t pitch) {
    if (!ctx || !d_field) return VD_ERR_INVALID;
    vd_batch* b = ctx->b;
    if ((long long)pitch < b->desc[0].uLx) return VD_ERR_INVALID;
    const long long p = (long long)pitch;
    std::vector<int> act{0};
    vd_status r = push_fields(b, act, &d_field, &p);
    if (r) return r;
    return run_all(b);
}

vd_status vd_push_frame_host(vd_ctx* ctx, const float* h_field, size_t pitch) {
    if (!ctx || !h_field) return VD_ERR_INVALID;
    vd_batch* b = ctx->b;
    const InstDesc& D = b->desc[0];
    if ((long long)pitch < D.uLx) return VD_ERR_INVALID;
    if (!b->d_host_field) {
        b->d_host_field = b->mem.alloc<float>((long long)D.uLx * D.uLy);
        if (!b->mem.ok) return VD_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy2DAsync(b->d_host_field, sizeof(float) * D.uLx, h_field, sizeof(float) * pitch,
                                      sizeof(float) * D.uLx, D.uLy, cudaMemcpyHostToDevice, b->s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
    return vd_push_frame(ctx, b->d_host_field, D.uLx);
}

vd_status vd_get_changes(vd_ctx* ctx, vd_changes* out) { return ctx ? get_changes(ctx->b, 0, out) : VD_ERR_INVALID; }

vd_status vd_set_obstacles(vd_ctx* ctx, const uint8_t* h_mask, int64_t pitch) {
    return ctx ? set_obstacles(ctx->b, 0, h_mask, pitch) : VD_ERR_INVALID;
}

vd_status vd_batch_set_obstacles(vd_batch* b, int32_t i, const uint8_t* h_mask, int64_t pitch) {
    return set_obstacles(b, i, h_mask, pitch);
}

vd_status vd_get_counts(vd_ctx* ctx, int32_t* K, int32_t* n_edges, int64_t* frame_index) {
    if (!ctx) return VD_ERR_INVALID;
    return vd_batch_get_counts(ctx->b, 0, K, n_edges, frame_index);
}
vd_status vd_get_labels(vd_ctx* ctx, int32_t* out, int64_t cap, int64_t* n) {
    return ctx ? get_array(ctx->b, 0, 0, out, cap, n) : VD_ERR_INVALID;
}
vd_status vd_get_owners(vd_ctx* ctx, int32_t* out, int64_t cap, int64_t* n) {
    return ctx ? get_array(ctx->b, 0, 1, out, cap, n) : VD_ERR_INVALID;
}
vd_status vd_get_centroids_q10(vd_ctx* ctx, int32_t* out, int64_t cap, int64_t* n) {
    return ctx ? get_array(ctx->b, 0, 2, out, cap, n) : VD_ERR_INVALID;
}
vd_status vd_get_edges(vd_ctx* ctx, uint64_t* out, int64_t cap, int64_t* n) {
    return ctx ? get_array(ctx->b, 0, 3, out, cap, n) : VD_ERR_INVALID;
}
vd_status vd_get_match(vd_ctx* ctx, int32_t* phi, int64_t cap, int64_t* n) {
    return ctx ? get_array(ctx->b, 0, 4, phi, cap, n) : VD_ERR_INVALID;
}

vd_status vd_export_state(vd_ctx* ctx, void* buf, int64_t cap, int64_t* n_bytes) {
    return ctx ? export_state(ctx->b, 0, buf, cap, n_bytes) : VD_ERR_INVALID;
}
vd_status vd_import_state(vd_ctx* ctx, const void* buf, int64_t n_bytes) {
    return ctx ? import_state(ctx->b, 0, buf, n_bytes) : VD_ERR_INVALID;
}
vd_status vd_batch_export_state(vd_batch* b, int32_t i, void* buf, int64_t cap, int64_t* n_bytes) {
    return export_state(b, i, buf, cap, n_bytes);
}
vd_status vd_batch_import_state(vd_batch* b, int32_t i, const void* buf, int64_t n_bytes) {
    return import_state(b, i, buf, n_bytes);
}

vd_status vd_debug_hold_scan_flag(vd_ctx* ctx, int32_t kind, int64_t tile, int32_t spin_limit) {
    if (!ctx || kind < 0 || kind >= SCAN_KINDS || tile < -1 || spin_limit < 0) return VD_ERR_INVALID;
    vd_batch* b = ctx->b;
    struct {
        int kind, spin;
        long long tile;
    } v = {kind, spin_limit, tile + 1};
    static_assert(offsetof(Globals, dbg_spin) == offsetof(Globals, dbg_kind) + sizeof(int) &&
                      offsetof(Globals, dbg_tile) == offsetof(Globals, dbg_kind) + 2 * sizeof(int),
                  "debug fields of Globals must be contiguous");
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<char*>(b->P.g) + offsetof(Globals, dbg_kind), &v, sizeof(v),
                                    cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    return cuda_status(e);
}

namespace {
// the checked build's record of the last step (Globals::chk_id, chk_index)
vd_status check_info(vd_batch* b, int32_t* checked, int32_t* first_check, int64_t* index) {
    if (!b || !checked || !first_check || !index) return VD_ERR_INVALID;
    struct {
        int id, dbg;
        long long index;
    } v = {0, 0, 0};
    static_assert(offsetof(Globals, dbg_chk) == offsetof(Globals, chk_id) + sizeof(int) &&
                      offsetof(Globals, chk_index) == offsetof(Globals, chk_id) + 2 * sizeof(int),
                  "check fields of Globals must be contiguous");
    cudaError_t e = cudaStreamSynchronize(b->s);
    if (e == cudaSuccess)
        e = cudaMemcpy(&v, reinterpret_cast<char*>(b->P.g) + offsetof(Globals, chk_id), sizeof(v),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    *checked = VD_IS_CHECKED ? 1 : 0;
    *first_check = v.id;
    *index = v.index;
    return VD_OK;
}

vd_status force_check(vd_batch* b, int32_t id) {
    if (!b || id < 0 || id >= CHK_COUNT) return VD_ERR_INVALID;
    const int v = id;
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<char*>(b->P.g) + offsetof(Globals, dbg_chk), &v, sizeof(v),
                                    cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    return cuda_status(e);
}
}  // namespace

vd_status vd_debug_check_info(vd_ctx* ctx, int32_t* checked, int32_t* first_check, int64_t* index) {
    return ctx ? check_info(ctx->b, checked, first_check, index) : VD_ERR_INVALID;
}
vd_status vd_debug_force_check(vd_ctx* ctx, int32_t id) { return ctx ? force_check(ctx->b, id) : VD_ERR_INVALID; }
vd_status vd_batch_debug_check_info(vd_batch* b, int32_t* checked, int32_t* first_check, int64_t* index) {
    return check_info(b, checked, first_check, index);
}
vd_status vd_batch_debug_force_check(vd_batch* b, int32_t id) { return force_check(b, id); }

vd_status vd_batch_set_tuning(vd_batch* b, const vd_tuning* t) {
    if (!b || !t) return VD_ERR_INVALID;
    if (t->voronoi_patch < 0 || t->voronoi_patch >= VPATCH_COUNT || t->bucket_pct < 25 || t->bucket_pct > 400 ||
        t->ring0 < 0 || t->ring0 > 256 || t->graph_blocks < 0 || t->graph_blocks > 1)
        return VD_ERR_INVALID;
    for (InstDesc& D : b->desc) {
        D.bucket_pct = t->bucket_pct;
        D.ring0 = t->ring0;
    }
    cudaError_t e = cudaMemcpyAsync(b->P.desc, b->desc.data(), sizeof(InstDesc) * b->n, cudaMemcpyHostToDevice, b->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) return VD_ERR_CUDA;
    if (t->voronoi_patch != b->vpatch || t->graph_blocks != b->graph_inst) {
        b->vpatch = t->voronoi_patch;
        b->graph_inst = t->graph_blocks;
        if (b->graph) {   // the step launches another kernel: capture it again
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
    }
    return VD_OK;
}

vd_status vd_batch_get_tuning(vd_batch* b, vd_tuning* t) {
    if (!b || !t) return VD_ERR_INVALID;
    t->voronoi_patch = b->vpatch;
    t->bucket_pct = b->desc[0].bucket_pct;
    t->ring0 = b->desc[0].ring0;
    t->graph_blocks = b->graph_inst;
    return VD_OK;
}

vd_status vd_set_tuning(vd_ctx* ctx, const vd_tuning* t) { return ctx ? vd_batch_set_tuning(ctx->b, t) : VD_ERR_INVALID; }
vd_status vd_get_tuning(vd_ctx* ctx, vd_tuning* t) { return ctx ? vd_batch_get_tuning(ctx->b, t) : VD_ERR_INVALID; }

vd_status vd_batch_set_timing(vd_batch* b, int32_t enable) {
    if (!b) return VD_ERR_INVALID;
    b->timing = enable != 0;
    return VD_OK;
}

vd_status vd_batch_get_timing(vd_batch* b, double* stage_ms, int32_t cap, int32_t* n_stages,
                              int64_t* n_kernel_launches, int64_t* n_steps) {
    if (!b) return VD_ERR_INVALID;
    if (cudaStreamSynchronize(b->s) != cudaSuccess) return VD_ERR_CUDA;
    if (n_stages) *n_stages = N_STAGES;
    if (n_kernel_launches) *n_kernel_launches = b->launches;
    if (n_steps) *n_steps = b->frames_pushed;
    double acc[N_STAGES] = {};
    const int per = N_STAGES + 1;
    for (int g = 0; g + per <= b->ev_used; g += per) {
        for (int k = 0; k < N_STAGES; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, b->ev_pool[g + k], b->ev_pool[g + k + 1]) == cudaSuccess) acc[k] += ms;
        }
    }
    b->ev_used = 0;
    if (stage_ms) {
        if (cap < N_STAGES) return VD_ERR_CAPACITY;
        for (int k = 0; k < N_STAGES; ++k) stage_ms[k] = acc[k];
    }
    return VD_OK;
}

vd_status vd_set_timing(vd_ctx* ctx, int32_t enable) {
    return ctx ? vd_batch_set_timing(ctx->b, enable) : VD_ERR_INVALID;
}

vd_status vd_get_timing(vd_ctx* ctx, double* stage_ms, int32_t cap, int32_t* n_stages,
                        int64_t* n_kernel_launches, int64_t* n_frames) {
    return ctx ? vd_batch_get_timing(ctx->b, stage_ms, cap, n_stages, n_kernel_launches, n_frames) : VD_ERR_INVALID;
}

const char* vd_stage_name(int32_t stage) {
    if (stage < 0 || stage >= N_STAGES) return "";
    return STAGE_NAMES[stage];
}

vd_status vd_destroy(vd_ctx* ctx) {
    if (!ctx) return VD_ERR_INVALID;
    vd_status r = vd_batch_destroy(ctx->b);
    delete ctx;
    return r;
}

vd_status vd_batch_create(const vd_config* cfgs, int32_t n, vd_batch** out) {
    vd_status r = create_batch(cfgs, n, out);
    if (!r) (*out)->use_graph = (cfgs[0].stream != nullptr);
    return r;
}

vd_status vd_batch_create_sequence(const vd_config* cfg, int32_t n_frames, vd_batch** out) {
    if (!cfg || n_frames < 1 || !out) return VD_ERR_INVALID;
    std::vector<vd_config> cfgs(n_frames, *cfg);
    vd_status r = create_batch(cfgs.data(), n_frames, out, true);
    if (!r) (*out)->use_graph = (cfg->stream != nullptr);
    return r;
}

vd_status vd_batch_push(vd_batch* b, const float* const* d_fields) {
    if (!b || !d_fields) return VD_ERR_INVALID;
    std::vector<int> act(b->n);
    std::vector<long long> pitch(b->n);
    for (int i = 0; i < b->n; ++i) {
        act[i] = i;
        pitch[i] = b->desc[i].uLx;
    }
    vd_status r = push_fields(b, act, d_fields, pitch.data());
    if (r) return r;
    return run_all(b);
}

vd_status vd_batch_stage_host(vd_batch* b, const float* const* h_fields) {
    if (!b || !h_fields) return VD_ERR_INVALID;
    for (int i = 0; i < b->n; ++i)
        if (!h_fields[i]) return VD_ERR_INVALID;
    if (!b->cs) {
        if (cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess) return VD_ERR_CUDA;
        for (int k = 0; k < 2; ++k)
            if (cudaEventCreateWithFlags(&b->ev_staged[k], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_read[k], cudaEventDisableTiming) != cudaSuccess)
                return VD_ERR_CUDA;
    }
    const int k = b->stage_next;
    if (b->d_stage[k].empty()) {
        // one allocation per buffer set: instance i's frame follows instance i-1's
        long long total = 0;
        for (int i = 0; i < b->n; ++i) total += (long long)b->desc[i].uLx * b->desc[i].uLy;
        float* base = b->mem.alloc<float>(total);
        if (!b->mem.ok) return VD_ERR_OOM;
        b->d_stage[k].resize(b->n);
        for (int i = 0; i < b->n; ++i) {
            b->d_stage[k][i] = base;
            base += (long long)b->desc[i].uLx * b->desc[i].uLy;
        }
    }
    // the step that last read this buffer must be done with it
    if (b->read_pending[k] && cudaStreamWaitEvent(b->cs, b->ev_read[k], 0) != cudaSuccess) return VD_ERR_CUDA;
    // host frames that follow each other in memory go in one copy; adjacent
    // frames from different host allocations make the runtime refuse the
    // merged copy (a non-sticky argument error), and they are copied one by one
    for (int i = 0; i < b->n;) {
        size_t bytes = sizeof(float) * (size_t)b->desc[i].uLx * b->desc[i].uLy;
        int j = i + 1;
        while (j < b->n && h_fields[j] == h_fields[i] + bytes / sizeof(float)) {
            bytes += sizeof(float) * (size_t)b->desc[j].uLx * b->desc[j].uLy;
            ++j;
        }
        if (cudaMemcpyAsync(b->d_stage[k][i], h_fields[i], bytes, cudaMemcpyHostToDevice, b->cs) != cudaSuccess) {
            if (j == i + 1) return VD_ERR_CUDA;
            cudaGetLastError();
            for (int m = i; m < j; ++m) {
                const size_t bm = sizeof(float) * (size_t)b->desc[m].uLx * b->desc[m].uLy;
                if (cudaMemcpyAsync(b->d_stage[k][m], h_fields[m], bm, cudaMemcpyHostToDevice, b->cs) != cudaSuccess)
                    return VD_ERR_CUDA;
            }
        }
        i = j;
    }
    if (cudaEventRecord(b->ev_staged[k], b->cs) != cudaSuccess) return VD_ERR_CUDA;
    b->staged = k;
    b->stage_next = k ^ 1;
    return VD_OK;
}

vd_status vd_batch_push_staged(vd_batch* b) {
    if (!b) return VD_ERR_INVALID;
    if (b->staged < 0) return VD_ERR_STATE;
    const int k = b->staged;
    if (cudaStreamWaitEvent(b->s, b->ev_staged[k], 0) != cudaSuccess) return VD_ERR_CUDA;
    vd_status r = vd_batch_push(b, b->d_stage[k].data());
    if (r) return r;
    if (cudaEventRecord(b->ev_read[k], b->s) != cudaSuccess) return VD_ERR_CUDA;
    b->read_pending[k] = true;
    b->staged = -1;
    return VD_OK;
}

vd_status vd_batch_push_host(vd_batch* b, const float* const* h_fields) {
    vd_status r = vd_batch_stage_host(b, h_fields);
    return r ? r : vd_batch_push_staged(b);
}

vd_status vd_batch_get_changes_all(vd_batch* b, vd_batch_changes* out) {
    if (!b || !out) return VD_ERR_INVALID;
    vd_status r = ensure_changes(b);
    if (r) return r;
    const int n = b->n;
    const long long nb = b->h_off[3 * n], na = b->h_off[3 * n + 1], nk = b->h_off[3 * n + 2];
    out->total_breaking = nb;
    out->total_arising = na;
    out->total_active = nk;
    for (int j = 0; j < n; ++j) {
        const InstState& st = b->h_st[j];
        const vd_status sj = st.frame == 0 ? VD_ERR_STATE : err_status(st);
        const bool ok = sj == VD_OK;
        if (out->status) out->status[j] = sj;
        if (out->n_prev) out->n_prev[j] = ok ? st.rep_K_prev : 0;
        if (out->n_now) out->n_now[j] = ok ? st.K : 0;
        if (out->n_breaking) out->n_breaking[j] = ok ? st.n_break : 0;
        if (out->n_arising) out->n_arising[j] = ok ? st.n_arise : 0;
    }
    if ((out->breaking && out->cap_breaking < nb) || (out->breaking_prev && out->cap_breaking < nb) ||
        (out->arising && out->cap_arising < na) || (out->active && out->cap_active < nk))
        return VD_ERR_CAPACITY;
    const size_t u8 = sizeof(unsigned long long);
    if (out->breaking) r = copy_from_host(out->breaking, b->h_chg, u8 * nb);
    if (!r && out->breaking_prev) r = copy_from_host(out->breaking_prev, b->h_chg + nb, u8 * nb);
    if (!r && out->arising) r = copy_from_host(out->arising, b->h_chg + 2 * nb, u8 * na);
    if (!r && out->active) r = copy_from_host(out->active, b->h_act, nk);
    return r;
}

vd_status vd_batch_push_subset(vd_batch* b, const int32_t* active, int32_t n_active, const float* const* d_fields) {
    if (!b || !active || !d_fields || n_active < 0 || n_active > b->n) return VD_ERR_INVALID;
    if (b->sequence) return VD_ERR_INVALID;   // a frame sequence always advances as a whole
    if (n_active == 0) return VD_OK;
    std::vector<int> act(active, active + n_active);
    std::vector<char> seen(b->n, 0);
    std::vector<long long> pitch(n_active);
    for (int a = 0; a < n_active; ++a) {
        if (act[a] < 0 || act[a] >= b->n || seen[act[a]]) return VD_ERR_INVALID;
        seen[act[a]] = 1;
        pitch[a] = b->desc[act[a]].uLx;
    }
    if (n_active == b->n) {
        bool ordered = true;
        for (int a = 0; a < n_active; ++a) ordered &= (act[a] == a);
        if (ordered) return vd_batch_push(b, d_fields);
    }
    vd_status r = push_fields(b, act, d_fields, pitch.data());
    if (r) return r;
    build_table(b, act, b->sub, false);
    enqueue_step(b, make_launch(b, b->sub), false);
    b->frames_pushed += 1;
    return step_status(b);
}

vd_status vd_batch_get_changes(vd_batch* b, int32_t i, vd_changes* out) { return get_changes(b, i, out); }
vd_status vd_batch_get_labels(vd_batch* b, int32_t i, int32_t* out, int64_t cap, int64_t* n) {
    return get_array(b, i, 0, out, cap, n);
}
vd_status vd_batch_get_owners(vd_batch* b, int32_t i, int32_t* out, int64_t cap, int64_t* n) {
    return get_array(b, i, 1, out, cap, n);
}
vd_status vd_batch_get_centroids_q10(vd_batch* b, int32_t i, int32_t* out, int64_t cap, int64_t* n) {
    return get_array(b, i, 2, out, cap, n);
}
vd_status vd_batch_get_edges(vd_batch* b, int32_t i, uint64_t* out, int64_t cap, int64_t* n) {
    return get_array(b, i, 3, out, cap, n);
}

vd_status vd_batch_get_counts(vd_batch* b, int32_t i, int32_t* K, int32_t* n_edges, int64_t* frame_index) {
    InstState st;
    vd_status r = read_state(b, i, &st);
    if (r) return r;
    if (K) *K = st.K;
    if (n_edges) *n_edges = st.E;
    if (frame_index) *frame_index = st.frame - 1;
    return err_status(st);
}

vd_status vd_batch_destroy(vd_batch* b) {
    if (!b) return VD_ERR_INVALID;
    cudaStreamSynchronize(b->s);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    cudaFree(b->d_chg);
    cudaFreeHost(b->h_chg);
    cudaFree(b->d_act);
    cudaFreeHost(b->h_act);
    cudaFree(b->d_off);
    cudaFreeHost(b->h_off);
    if (b->cs) {
        cudaStreamSynchronize(b->cs);
        cudaStreamDestroy(b->cs);
    }
    if (b->s2) {
        cudaStreamSynchronize(b->s2);
        cudaStreamDestroy(b->s2);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    for (int k = 0; k < 2; ++k) {
        if (b->ev_staged[k]) cudaEventDestroy(b->ev_staged[k]);
        if (b->ev_read[k]) cudaEventDestroy(b->ev_read[k]);
    }
    b->mem.release();
    delete b;
    return VD_OK;
}

}  // extern "C"
