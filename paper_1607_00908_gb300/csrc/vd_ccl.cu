// Bubble identification (Section 3.1 of the paper): threshold, periodic
// 4-connected labelling with canonical ids, sizes and centres of mass in
// 1/1024-site fixed point, the centroid bucket grid, and the run-label pass
// that also builds the past/now overlap histogram (Section 3.2.3).
//
// Labelling works on 64 x 32 tiles. The threshold pass reads the field once
// (coalesced 16-byte loads, two tile rows per warp load) and stores the
// foreground bits (1 bit per site); pass A reads a tile's row words, runs a
// union-find over its runs in shared memory and emits one "piece" per
// tile-local component with its size and coordinate sums relative to its
// first site, plus the piece ids along the four tile borders. Pieces are then merged across tile borders (periodic) by
// a global union-find whose root is the piece with the smallest first site, so
// the root of every bubble is the bubble's smallest linear index; bubble ids
// are the ranks of those roots (a scan of root counts per 256-site group of a
// row, then the root bits before each root in its group). Labels are kept
// per run (a 64-site tile row holds at most 32 runs): pass A records each
// run's piece, the run-label pass turns pieces into bubble ids, and per-site
// labels are expanded from the foreground bits and run labels on request.
#include "vd_internal.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// tile-local union-find in shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ int uf_find(volatile int* p, int x) {
    int y = p[x];
    while (y != x) {
        x = y;
        y = p[x];
    }
    return x;
}

// lock-free union by smaller index (the root of a set is its smallest index)
__device__ __forceinline__ void uf_union(int* p, int a, int b) {
    bool done;
    do {
        a = uf_find(p, a);
        b = uf_find(p, b);
        if (a < b) {
            int old = atomicMin(&p[b], a);
            done = (old == b);
            b = old;
        } else if (b < a) {
            int old = atomicMin(&p[a], b);
            done = (old == a);
            a = old;
        } else {
            done = true;
        }
    } while (!done);
}

// ---------------------------------------------------------------------------
// Warp-per-tile labelling. A 64 x 32 tile is handled by one warp: lane r owns
// tile row r, whose 64 foreground bits live in one 64-bit mask. Runs of a row
// are numbered left to right; run j of row r has id r*32 + j, so ids follow
// raster order and the smallest id of a component is its first site.
// ---------------------------------------------------------------------------
constexpr int RUNS = TRUNS;     // run ids per tile

__device__ __forceinline__ unsigned long long run_starts(unsigned long long m) { return m & ~(m << 1); }
__device__ __forceinline__ unsigned long long upto(int c) { return c == 63 ? ~0ull : ((2ull << c) - 1ull); }
// index of the run of row mask m (starts S) that contains column c (bit c set)
__device__ __forceinline__ int run_index(unsigned long long S, int c) { return __popcll(S & upto(c)) - 1; }
__device__ __forceinline__ int run_length(unsigned long long m, int c) {
    const unsigned long long inv = ~(m >> c);
    return inv ? __ffsll(inv) - 1 : 64;   // all ones only when c == 0
}

// Run id r*32 + j is stored at r*32 + (j ^ r): lanes that own different rows
// touch different shared-memory banks.
__device__ __forceinline__ int SW(int id) { return id ^ ((id >> 5) & 31); }

__device__ __forceinline__ int rfind(volatile int* p, int x) {
    int y = p[SW(x)];
    while (y != x) {
        x = y;
        y = p[SW(x)];
    }
    return x;
}

// root of run x, splitting the path on the way (each visited run is pointed at
// its grandparent). Used only while unions run: concurrent splits and unions
// store ancestors of non-roots, so the sets stay intact. The flatten that
// follows must not run concurrently with splits, which could replace a
// flattened root by an intermediate ancestor.
__device__ __forceinline__ int rfind_split(volatile int* p, int x) {
    int y = p[SW(x)];
    while (y != x) {
        const int z = p[SW(y)];
        if (z != y) p[SW(x)] = z;
        x = y;
        y = z;
    }
    return x;
}

// lock-free union by smaller run id on the swizzled parent array
__device__ __forceinline__ void runion(int* p, int a, int b) {
    bool done;
    do {
        a = rfind_split(p, a);
        b = rfind_split(p, b);
        if (a < b) {
            const int old = atomicMin(&p[SW(b)], a);
            done = (old == b);
            b = old;
        } else if (b < a) {
            const int old = atomicMin(&p[SW(a)], b);
            done = (old == a);
            a = old;
        } else {
            done = true;
        }
    } while (!done);
}

struct UfSmem {                  // one warp's tile: row masks and union-find over runs
    unsigned long long m[TH];
    int par[RUNS];               // swizzled: parent of run id k at par[SW(k)]
    unsigned char col[RUNS];     // swizzled: start column of each run (pass A: then the run's
                                 // piece index within the tile, in a tile of at most PCAP pieces)
};
// piece id of run `id` in a tile of more than PCAP pieces, after pass A has
// stored -2 - (piece id) in the parent slot of every root; *root = the run id
// of its root
__device__ __forceinline__ int run_piece(const UfSmem& T, int id, int* root) {
    const int v = T.par[SW(id)];
    if (v < 0) {
        *root = id;
        return -2 - v;
    }
    *root = v;
    return -2 - T.par[SW(v)];
}

// The pairs (j, ju) of touching runs between row r (run j) and row r-1 (run
// ju) of a tile, for lane r > 0; f(j, ju) is called for each. 4-connectivity
// joins runs that share a column (one pair per segment of m & mu, in column
// order); with 8-connectivity a run of row r-1 widened by one column on each
// side joins every run of row r it meets.
template <class F>
__device__ __forceinline__ void touching_pairs(unsigned long long m, unsigned long long mu, bool conn8, F&& f) {
    const unsigned long long S = run_starts(m), Su = run_starts(mu);
    if (!conn8) {
        unsigned long long os = run_starts(m & mu);
        while (os) {
            const int c = __ffsll(os) - 1;
            os &= os - 1;
            f(run_index(S, c), run_index(Su, c));
        }
    } else {
        unsigned long long tu = Su;
        int ju = 0;
        while (tu) {
            const int cu = __ffsll(tu) - 1;
            tu &= tu - 1;
            const int len = run_length(mu, cu);
            const unsigned long long ru = (len >= 64 ? ~0ull : ((1ull << len) - 1ull)) << cu;
            unsigned long long hs = run_starts(m & (ru | (ru << 1) | (ru >> 1)));
            while (hs) {
                const int c = __ffsll(hs) - 1;
                hs &= hs - 1;
                f(run_index(S, c), ju);
            }
            ++ju;
        }
    }
}

// Union-find over the runs of a tile; lane r owns row r, m = its row mask.
// On return the parent slot of every run holds its root, the smallest run id
// of its component (so roots follow raster order).
//  1. every run of row r > 0 takes as parent the first run of row r-1 it
//     touches: a forest in which each parent lies one row up, so each tree's
//     root is its smallest id;
//  2. pointer jumping (every run's parent becomes its grandparent, rounds
//     separated by warp barriers, until no parent changes) makes every
//     parent a tree root in about log2(rows) rounds, where a find per run
//     would walk one row per step;
//  3. the remaining touching pairs join their trees (union by smaller root);
//  4. a find per run (tree root, then the few joined roots) flattens.
// Reads in step 2 may see another lane's newer value, which is an ancestor
// too, so the rounds only end sooner.
__device__ void warp_runs_uf(UfSmem& T, unsigned long long m, bool conn8) {
    const int r = threadIdx.x & 31;
    const unsigned long long S = run_starts(m);
    const int nr = __popcll(S);
    {
        unsigned long long t = S;
        int j = 0;
        while (t) {
            const int c = __ffsll(t) - 1;
            t &= t - 1;
            T.par[SW(r * 32 + j)] = r * 32 + j;
            T.col[SW(r * 32 + j)] = (unsigned char)c;
            ++j;
        }
    }
    const unsigned long long mu = __shfl_up_sync(0xffffffffu, m, 1);
    unsigned linked = 0;    // runs of this row with a parent in row r-1
    bool more = false;      // a run of this row touches a second run above
    if (r > 0) {
        touching_pairs(m, mu, conn8, [&](int j, int ju) {
            if ((linked >> j) & 1u) {
                more = true;
            } else {
                linked |= 1u << j;
                T.par[SW(r * 32 + j)] = (r - 1) * 32 + ju;
            }
        });
    }
    for (;;) {
        __syncwarp();
        bool changed = false;
        unsigned t = linked;
        while (t) {
            const int x = r * 32 + __ffs(t) - 1;
            t &= t - 1;
            const int p = T.par[SW(x)];
            const int pp = T.par[SW(p)];
            if (pp != p) {
                T.par[SW(x)] = pp;
                changed = true;
            }
        }
        if (!__any_sync(0xffffffffu, changed)) break;
    }
    __syncwarp();
    if (more) {
        unsigned seen = 0;
        touching_pairs(m, mu, conn8, [&](int j, int ju) {
            if ((seen >> j) & 1u) runion(T.par, r * 32 + j, (r - 1) * 32 + ju);
            seen |= 1u << j;
        });
    }
    __syncwarp();
    for (int j = 0; j < nr; ++j) T.par[SW(r * 32 + j)] = rfind(T.par, r * 32 + j);
    __syncwarp();
}

// mask (over run indices) of this lane's root runs, and the exclusive count of
// roots in rows above (raster order); *total = roots in the tile
__device__ __forceinline__ unsigned warp_roots(const UfSmem& T, unsigned long long m, int* base, int* total) {
    const int r = threadIdx.x & 31;
    const int nr = __popcll(run_starts(m));
    unsigned R = 0;
    for (int j = 0; j < nr; ++j)
        if (T.par[SW(r * 32 + j)] == r * 32 + j) R |= 1u << j;
    const int cnt = __popc(R);
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (r >= o) inc += y;
    }
    *base = inc - cnt;
    *total = __shfl_sync(0xffffffffu, inc, 31);
    return R;
}

// Run tables (piece id and bubble label of every run) are kept per labelling
// tile in RUNS slots, packed in row-major order: the runs of row r start at
// slot run_row_base(r) = the number of runs in rows 0..r-1 of the tile, so a
// tile's runs fill a contiguous prefix of its slots (few DRAM sectors per
// tile). Lane r of a warp holding the tile's row masks gets its row's base by
// a prefix sum of the rows' run counts.
__device__ __forceinline__ int run_row_base(int nr) {
    const int lane = threadIdx.x & 31;
    int inc = nr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    return inc - nr;
}

// row masks of a tile from stored foreground bits `fg` (lane r -> row r)
__device__ __forceinline__ unsigned long long load_row_mask(const unsigned* fg, const InstDesc& D, int x0, int y0) {
    const int y = y0 + (threadIdx.x & 31);
    unsigned long long m = 0;
    if (y < D.Ly) {
        const unsigned* row = fg + D.word_off + (long long)y * D.wpr;
        const int wx = x0 >> 5;
        m = row[wx];
        if (wx + 1 < D.wpr) m |= (unsigned long long)row[wx + 1] << 32;
    }
    return m;
}

__device__ __forceinline__ bool is_fg(float v, float thr, int pol) {
    return pol > 0 ? (v > thr) : (v < thr);
}

constexpr int CCL_WARPS = 4;    // tiles per block in pass A
constexpr int PCAP = 32;        // pieces per tile summed in shared memory

// Threshold (Section 3.1) of a 64 x 32 tile, read straight from the field
// with coalesced 16-byte loads: one warp load covers two tile rows (lanes
// 0-15 row 2s, lanes 16-31 row 2s+1, four columns per lane); each 8-lane group
// holds one 32-bit word of a row, or-reduced across the warp, and the row's
// lane keeps the 64-bit mask. Eight row pairs are read at a time. Bit i of
// row y's mask is site (x0 + i, y0 + y); rows at or past nrow and columns at
// or past ncol are 0. Rows that are not 16-byte aligned, or a tile cut by the
// domain edge, take scalar loads.
__device__ __forceinline__ unsigned long long threshold_tile(const float* f0, long long pitch, int nrow, int ncol,
                                                             float thr, int pol) {
    const int lane = threadIdx.x & 31;
    const int hr = lane >> 4, c = 4 * (lane & 15), g = lane >> 3, sh = 4 * (lane & 7);
    const bool vec = ncol == TW && ((reinterpret_cast<uintptr_t>(f0) | (uintptr_t)(pitch * 4)) & 15u) == 0;
    const unsigned cm = ncol >= c + 4 ? 0xFu : (ncol > c ? (1u << (ncol - c)) - 1u : 0u);
    unsigned long long my_m = 0;
#pragma unroll
    for (int sb = 0; sb < TH / 2; sb += 8) {
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int y = 2 * (sb + i) + hr;
            if (y < nrow) {
                const float* p = f0 + (long long)y * pitch + c;
                if (vec) {
                    v[i] = __ldcs(reinterpret_cast<const float4*>(p));
                } else {
                    if (cm & 1u) v[i].x = __ldcs(p);
                    if (cm & 2u) v[i].y = __ldcs(p + 1);
                    if (cm & 4u) v[i].z = __ldcs(p + 2);
                    if (cm & 8u) v[i].w = __ldcs(p + 3);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int y = 2 * (sb + i) + hr;
            const unsigned nib = y < nrow ? ((unsigned)is_fg(v[i].x, thr, pol) | ((unsigned)is_fg(v[i].y, thr, pol) << 1) |
                                             ((unsigned)is_fg(v[i].z, thr, pol) << 2) |
                                             ((unsigned)is_fg(v[i].w, thr, pol) << 3)) & cm
                                          : 0u;
            const unsigned part = nib << sh;
            const unsigned r0 = __reduce_or_sync(0xffffffffu, g == 0 ? part : 0u);
            const unsigned r1 = __reduce_or_sync(0xffffffffu, g == 1 ? part : 0u);
            const unsigned r2 = __reduce_or_sync(0xffffffffu, g == 2 ? part : 0u);
            const unsigned r3 = __reduce_or_sync(0xffffffffu, g == 3 ? part : 0u);
            if (lane == 2 * (sb + i)) my_m = ((unsigned long long)r1 << 32) | r0;
            if (lane == 2 * (sb + i) + 1) my_m = ((unsigned long long)r3 << 32) | r2;
        }
    }
    return my_m;
}

// ---------------------------------------------------------------------------
// Threshold pass (Section 3.1): one warp per 64 x 32 labelling tile reads the
// field with coalesced loads and stores the tile's foreground words (kept for
// the labelling, the run-label pass and the next frame). Alone, it streams the
// field at the HBM rate; the union-find that follows reads the words from L2.
// ---------------------------------------------------------------------------
constexpr int THR_WARPS = 4;

__global__ __launch_bounds__(32 * THR_WARPS, 8) void k_threshold(Pools P, StepTable T) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * THR_WARPS + (threadIdx.x >> 5);
    if (b >= T.tileA_pre[T.n_act]) return;
    const int a = warp_seg_of_int(T.tileA_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileA_pre[a];
    const int x0 = (t % D.ntx) * TW, y0 = (t / D.ntx) * TH;
    // the field covers the domain only (a bounded axis runs with twice its
    // length; the second half is never a bubble)
    unsigned long long m = threshold_tile(S.field + (long long)y0 * S.pitch + x0, S.pitch,
                                          min(TH, min(D.Ly, D.uLy) - y0), min(TW, D.uLx - x0), D.thr, D.pol);
    const int y = y0 + lane;
    if (y < D.Ly) {
        const int n = min(TW, D.Lx - x0);
        unsigned* row = P.fgbits[S.slot ^ 1] + D.word_off + (long long)y * D.wpr + (x0 >> 5);
        if (D.masked) {   // obstacle sites are never in a bubble
            const unsigned* ob = P.obst + D.word_off + (long long)y * D.wpr + (x0 >> 5);
            unsigned long long om = ob[0];
            if (n > 32) om |= (unsigned long long)ob[1] << 32;
            m &= ~om;
        }
        row[0] = (unsigned)m;
        if (n > 32) row[1] = (unsigned)(m >> 32);
    }
}

// ---------------------------------------------------------------------------
// Pass A: union-find over runs + pieces + borders (one warp per tile)
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(32 * CCL_WARPS, 9) void k_ccl_tiles(Pools P, StepTable T) {
    pdl_enter();
    __shared__ UfSmem s_tile[CCL_WARPS];
    __shared__ int4 s_pc[CCL_WARPS][PCAP];   // per piece: size, row sum, column sum, first site
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * CCL_WARPS + w;
    if (b >= T.tileA_pre[T.n_act]) return;
    UfSmem& TS = s_tile[w];
    const int a = warp_seg_of_int(T.tileA_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileA_pre[a];
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const int Lx = D.Lx, Ly = D.Ly;

    // 1. this tile's row masks, stored by the threshold pass (lane r: row r)
    const unsigned long long my_m = load_row_mask(P.fgbits[S.slot ^ 1], D, x0, y0);
    TS.m[lane] = my_m;

    // 2. union-find over runs
    warp_runs_uf(TS, my_m, D.conn8 != 0);

    // 3. pieces: the tile's roots in raster order are its pieces 0 .. m_tot-1,
    //    numbered in the piece pool from a base taken with one atomic add
    const unsigned long long S0 = run_starts(my_m);
    const int nr = __popcll(S0);
    int rbase, m_tot;
    const unsigned R = warp_roots(TS, my_m, &rbase, &m_tot);
    int pbase = 0;
    if (lane == 0) pbase = atomicAdd(&P.g->n_pieces, m_tot);
    const int ncols = min(TW, Lx - x0), nrows = min(TH, Ly - y0);
    int* bd = P.border + D.border_off + (long long)t * BORDER;
    const int rrow = run_row_base(nr);
    int* rp = P.rp + (long long)(D.tile_off + t) * RUNS + rrow;

    if (m_tot <= PCAP) {
        // A tile of at most PCAP pieces sums them in shared memory while the
        // atomic add is in flight: a root's parent slot takes -2 - (its local
        // index k), and per piece the size, the sums of row and of column over
        // its sites (tile coordinates) and its first site (row << 16 | column)
        // are kept; every run's start-column byte then takes its piece's k.
        int4* pc = s_pc[w];
        {
            unsigned rq = R;
            int k = rbase;
            while (rq) {
                const int id = SW(lane * 32 + __ffs(rq) - 1);
                rq &= rq - 1;
                pc[k] = make_int4(0, 0, 0, (lane << 16) | TS.col[id]);
                TS.par[id] = -2 - k;
                ++k;
            }
        }
        __syncwarp();
        {
            unsigned long long q = S0;
            for (int j = 0; j < nr; ++j) {
                const int c = __ffsll(q) - 1;
                q &= q - 1;
                const int id = SW(lane * 32 + j);
                const int v = TS.par[id];
                const int k = -2 - (v < 0 ? v : TS.par[SW(v)]);
                const int len = run_length(my_m, c);
                atomicAdd(&pc[k].x, len);
                atomicAdd(&pc[k].y, len * lane);
                atomicAdd(&pc[k].z, len * c + (len * (len - 1)) / 2);
                TS.col[id] = (unsigned char)k;
            }
        }
        __syncwarp();
        if (lane == 0) {
            if (pbase + m_tot > P.piece_cap) {
                atomicOr(&P.g->err, ERR_PIECE_CAP);
                atomicOr(&P.st[inst].err, ERR_PIECE_CAP);
                pbase = -1;
            }
            P.tile_pbase[D.tile_off + t] = pbase;
            P.tile_pcnt[D.tile_off + t] = m_tot;
        }
        pbase = __shfl_sync(0xffffffffu, pbase, 0);
        // 4. run -> piece table (for the run-label pass) and the piece records
        //    (coalesced; sums relative to the piece's first site)
        for (int j = 0; j < nr; ++j)
            if (vd_in(P, CHK_RUN_PIECE, rrow + j, RUNS)) rp[j] = pbase >= 0 ? pbase + TS.col[SW(lane * 32 + j)] : -1;
        if (pbase >= 0) {
            for (int k = lane; k < m_tot; k += 32) {
                const int pid = pbase + k;
                if (!vd_in(P, CHK_TILE_PIECES, pid, P.piece_cap)) continue;
                const int4 e = pc[k];
                const int fr = e.w >> 16, fc = e.w & 0xffff;
                P.p_q[pid] = (y0 + fr) * Lx + x0 + fc;
                P.p_inst[pid] = inst;
                P.p_n[pid] = e.x;
                P.p_sv[pid] = e.y - e.x * fr;
                P.p_su[pid] = e.z - e.x * fc;
                P.p_parent[pid] = pid;
                P.p_accn[pid] = 0;
                P.p_accx[pid] = 0;
                P.p_accy[pid] = 0;
            }
        }
        // 5. borders: [0,TH) left col, [TH,2TH) right col, [2TH,2TH+TW) top
        //    row, [.., +TW) bottom row: piece id of each site, or -1
        auto piece_at = [&](unsigned long long m, int ly, int lx) -> int {
            if (pbase < 0 || lx >= ncols || ly >= nrows || !((m >> lx) & 1ull)) return -1;
            return pbase + TS.col[SW(ly * 32 + run_index(run_starts(m), lx))];
        };
        const unsigned long long mt = TS.m[0], mb = TS.m[nrows - 1];
        bd[lane] = piece_at(my_m, lane, 0);
        bd[TH + lane] = piece_at(my_m, lane, ncols - 1);
        bd[2 * TH + lane] = piece_at(mt, 0, lane);
        bd[2 * TH + 32 + lane] = piece_at(mt, 0, lane + 32);
        bd[2 * TH + TW + lane] = piece_at(mb, nrows - 1, lane);
        bd[2 * TH + TW + 32 + lane] = piece_at(mb, nrows - 1, lane + 32);
        return;
    }

    // A tile of more pieces: the records are initialised by their roots' lanes
    // and the sums added with global atomics, runs of one piece merged across
    // the warp first; a root's parent slot takes -2 - (its piece id).
    if (lane == 0) {
        if (pbase + m_tot > P.piece_cap) {
            atomicOr(&P.g->err, ERR_PIECE_CAP);
            atomicOr(&P.st[inst].err, ERR_PIECE_CAP);
            pbase = -1;
        }
        P.tile_pbase[D.tile_off + t] = pbase;
        P.tile_pcnt[D.tile_off + t] = m_tot;
    }
    pbase = __shfl_sync(0xffffffffu, pbase, 0);
    {
        unsigned rq = R;
        int k = rbase;
        while (rq) {
            const int j = __ffs(rq) - 1;
            rq &= rq - 1;
            const int id = SW(lane * 32 + j);
            int pid = -1;
            if (pbase >= 0 && vd_in(P, CHK_TILE_PIECES, pbase + k, P.piece_cap)) {
                pid = pbase + k;
                P.p_q[pid] = (y0 + lane) * Lx + x0 + TS.col[id];
                P.p_inst[pid] = inst;
                P.p_n[pid] = 0;
                P.p_sv[pid] = 0;
                P.p_su[pid] = 0;
                P.p_parent[pid] = pid;
                P.p_accn[pid] = 0;
                P.p_accx[pid] = 0;
                P.p_accy[pid] = 0;
            }
            ++k;
            TS.par[id] = -2 - pid;
        }
    }
    __syncwarp();
    {
        const int maxnr = __reduce_max_sync(0xffffffffu, nr);
        unsigned long long q = S0;
        for (int j = 0; j < maxnr; ++j) {
            int pid = -1, len = 0, sv = 0, su = 0;
            if (j < nr) {
                const int c = __ffsll(q) - 1;
                q &= q - 1;
                len = run_length(my_m, c);
                int root;
                pid = run_piece(TS, lane * 32 + j, &root);
                sv = len * (lane - (root >> 5));
                su = len * (c - TS.col[SW(root)]) + (len * (len - 1)) / 2;
                if (vd_in(P, CHK_RUN_PIECE, rrow + j, RUNS)) rp[j] = pid;
            }
            const unsigned grp = __match_any_sync(0xffffffffu, pid);
            const int gn = __reduce_add_sync(grp, len);
            const int gsv = __reduce_add_sync(grp, sv);
            const int gsu = __reduce_add_sync(grp, su);
            if (pid >= 0 && lane == __ffs(grp) - 1) {
                atomicAdd(&P.p_n[pid], gn);
                atomicAdd(&P.p_sv[pid], gsv);
                atomicAdd(&P.p_su[pid], gsu);
            }
        }
    }
    auto piece_at = [&](unsigned long long m, int ly, int lx) -> int {
        if (lx >= ncols || ly >= nrows || !((m >> lx) & 1ull)) return -1;
        int root;
        return run_piece(TS, ly * 32 + run_index(run_starts(m), lx), &root);
    };
    const unsigned long long mt = TS.m[0], mb = TS.m[nrows - 1];
    bd[lane] = piece_at(my_m, lane, 0);
    bd[TH + lane] = piece_at(my_m, lane, ncols - 1);
    bd[2 * TH + lane] = piece_at(mt, 0, lane);
    bd[2 * TH + 32 + lane] = piece_at(mt, 0, lane + 32);
    bd[2 * TH + TW + lane] = piece_at(mb, nrows - 1, lane);
    bd[2 * TH + TW + 32 + lane] = piece_at(mb, nrows - 1, lane + 32);
}

// ---------------------------------------------------------------------------
// Global union-find over pieces (root = piece with the smallest first site)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pfind(int* par, int x) {
    for (;;) {
        const int p = __ldcg(par + x);
        if (p == x) return x;
        const int gp = __ldcg(par + p);
        if (gp != p) par[x] = gp;   // path halving; gp is an ancestor of x
        x = p;
    }
}

// root of piece x without writing (for the flatten pass): there a halving
// store into another piece's slot could land after that piece's thread has
// written its final root, leaving an intermediate piece in the slot
__device__ __forceinline__ int pfind_ro(const int* par, int x) {
    for (;;) {
        const int p = __ldcg(par + x);
        if (p == x) return x;
        x = p;
    }
}

__device__ __forceinline__ void punion(const Pools& P, int a, int b) {
    if (!vd_in(P, CHK_MERGE_PARENT, a, P.piece_cap) || !vd_in(P, CHK_MERGE_PARENT, b, P.piece_cap)) return;
    for (;;) {
        a = pfind(P.p_parent, a);
        b = pfind(P.p_parent, b);
        if (a == b) return;
        const int qa = P.p_q[a], qb = P.p_q[b];
        if (qa > qb) { const int t = a; a = b; b = t; }
        if (atomicCAS(&P.p_parent[b], b, a) == b) return;
    }
}

// One warp per labelling tile: lane j joins row j of the tile's right edge
// with the left edge of the tile to its right, and columns j and 32 + j of
// its bottom edge with the top edge of the tile below (both periodic). A
// position whose piece pair equals the previous position's on the same edge
// adds nothing and is skipped. With 8-connectivity a position also joins the
// diagonal neighbours across its edge (the next row / column), and the right
// edge's first and last rows join across the tile corners.
constexpr int MERGE_WARPS = 8;

__global__ __launch_bounds__(32 * MERGE_WARPS) void k_ccl_merge(Pools P, StepTable T) {
    pdl_enter();
    __shared__ int s_pre[SEG_CACHE];
    const int* tpre = seg_table(T.tileA_pre, T.n_act, s_pre);
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * MERGE_WARPS + (threadIdx.x >> 5);
    if (b >= tpre[T.n_act]) return;
    const int a = seg_of_int(tpre, T.n_act, b);
    const InstDesc& D = P.desc[T.act[a]];
    const int t = b - tpre[a];
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int* bd = P.border + D.border_off;
    const int* bt = bd + (long long)t * BORDER;
    const int* br = bd + (long long)(ty * D.ntx + (tx + 1) % D.ntx) * BORDER;      // tile to the right
    const int* bb = bd + (long long)(((ty + 1) % D.nty) * D.ntx + tx) * BORDER;    // tile below
    const int nrows = min(TH, D.Ly - ty * TH), ncols = min(TW, D.Lx - tx * TW);
    const bool c8 = D.conn8 != 0;

    // right edge: row `lane`
    {
        const int pa = bt[TH + lane], pb = br[lane];
        const int ppa = __shfl_up_sync(0xffffffffu, pa, 1), ppb = __shfl_up_sync(0xffffffffu, pb, 1);
        if (pa >= 0 && pb >= 0 && !(lane > 0 && ppa == pa && ppb == pb)) punion(P, pa, pb);
        if (c8) {
            if (lane + 1 < nrows) {
                const int qa = bt[TH + lane + 1], qb = br[lane + 1];
                if (pa >= 0 && qb >= 0 && pa != qb) punion(P, pa, qb);
                if (qa >= 0 && pb >= 0 && qa != pb) punion(P, qa, pb);
            }
            if (lane == nrows - 1 && pa >= 0) {   // bottom-right corner: top-left site of the tile below-right
                const int v = bd[(long long)(((ty + 1) % D.nty) * D.ntx + (tx + 1) % D.ntx) * BORDER + 0];
                if (v >= 0 && v != pa) punion(P, pa, v);
            }
            if (lane == 0 && pa >= 0) {           // top-right corner: bottom-left site of the tile above-right
                const int tyu = (ty + D.nty - 1) % D.nty;
                const int nru = min(TH, D.Ly - tyu * TH);
                const int v = bd[(long long)(tyu * D.ntx + (tx + 1) % D.ntx) * BORDER + nru - 1];
                if (v >= 0 && v != pa) punion(P, pa, v);
            }
        }
    }
    // bottom edge: columns `lane` and 32 + `lane`
    int lpa = -1, lpb = -1;   // pair of column 31, carried to column 32
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = 32 * h + lane;
        const int pa = bt[2 * TH + TW + k], pb = bb[2 * TH + k];
        int ppa = __shfl_up_sync(0xffffffffu, pa, 1), ppb = __shfl_up_sync(0xffffffffu, pb, 1);
        if (lane == 0) {
            ppa = lpa;
            ppb = lpb;
        }
        const bool repeat = (k > 0) && ppa == pa && ppb == pb;
        if (pa >= 0 && pb >= 0 && !repeat) punion(P, pa, pb);
        if (c8 && k + 1 < ncols) {
            const int qa = bt[2 * TH + TW + k + 1], qb = bb[2 * TH + k + 1];
            if (pa >= 0 && qb >= 0 && pa != qb) punion(P, pa, qb);
            if (qa >= 0 && pb >= 0 && qa != pb) punion(P, qa, pb);
        }
        lpa = __shfl_sync(0xffffffffu, pa, 31);
        lpb = __shfl_sync(0xffffffffu, pb, 31);
    }
}

// root of each piece; roots are counted per instance and marked in the root
// bitmap. Every slot is written only by its own thread, with its root: a
// concurrent reader passing through it sees the old parent or the root, both
// ancestors, so each slot ends holding its root.
__global__ void k_ccl_flatten(Pools P) {
    pdl_enter();
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        const int r = pfind_ro(P.p_parent, pid);
        P.p_parent[pid] = r;
        if (r == pid) {
            const int inst = P.p_inst[pid];
            const InstDesc& D = P.desc[inst];
            const int q = P.p_q[pid];
            const int y = q / D.Lx, x = q - y * D.Lx;
            if (!vd_in(P, CHK_FGBITS, q, (long long)D.Lx * D.Ly)) continue;
            atomicOr(&P.rootbits[D.word_off + (long long)y * D.wpr + (x >> 5)], 1u << (x & 31));
            atomicAdd(&P.rgcnt[D.grp_off + (long long)y * D.gpr + (x >> 5) / RGW], 1);
            warp_add(&P.st[inst].K, 1);
        }
    }
}

// bubble ids of roots; exact coordinate sums relative to the bubble's first site
__global__ void k_comp_accum(Pools P) {
    pdl_enter();
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const int r = P.p_parent[pid];
        const int q = P.p_q[pid];
        const int yq = q / D.Lx, xq = q - yq * D.Lx;
        if (r == pid) {
            // rank = roots of earlier groups + earlier roots of this group
            const unsigned* row = P.rootbits + D.word_off + (long long)yq * D.wpr;
            const int wq = xq >> 5, w0 = wq - wq % RGW;
            int c = P.rankpre[D.grp_off + (long long)yq * D.gpr + wq / RGW] + __popc(row[wq] & ((1u << (xq & 31)) - 1u));
#pragma unroll
            for (int k = 0; k < RGW - 1; ++k)   // independent loads, issued together
                if (w0 + k < wq) c += __popc(row[w0 + k]);
            P.p_comp[pid] = c;
            if (c < D.comp_cap && vd_in(P, CHK_COMP_ID, c, D.comp_cap)) P.comp_root[D.comp_off + c] = pid;
        }
        const int qr = P.p_q[r];
        const int yr = qr / D.Lx, xr = qr - yr * D.Lx;
        const long long dx = wrap_ll(xq - xr, D.Lx), dy = wrap_ll(yq - yr, D.Ly);
        // every site of the piece lies in its tile: x - x_q in [umin, umax], y - y_q in [0, vmax]
        const int tx0 = (xq / TW) * TW, ty0 = (yq / TH) * TH;
        const long long umin = tx0 - xq, umax = min(tx0 + TW, D.Lx) - 1 - xq;
        const long long vmax = min(ty0 + TH, D.Ly) - 1 - yq;
        const long long hx = D.Lx / 2, hy = D.Ly / 2;
        const bool ok = (dx + umin >= -hx) && (dx + umax < D.Lx - hx) && (dy >= -hy) && (dy + vmax < D.Ly - hy);
        if (ok) {
            const long long nn = P.p_n[pid];
            atomicAdd((unsigned long long*)&P.p_accn[r], (unsigned long long)nn);
            atomicAdd((unsigned long long*)&P.p_accx[r], (unsigned long long)(nn * dx + P.p_su[pid]));
            atomicAdd((unsigned long long*)&P.p_accy[r], (unsigned long long)(nn * dy + P.p_sv[pid]));
        } else {
            const int w = warp_fetch_inc(&P.g->n_wide);
            if (vd_in(P, CHK_WIDE, w, P.piece_cap)) P.wide[w] = pid;
        }
    }
}

// exact per-site sums for pieces whose minimum image is not a single shift
// (one warp per piece; warps of a block work on different pieces)
constexpr int WIDE_WARPS = 4;
__global__ __launch_bounds__(32 * WIDE_WARPS) void k_comp_wide(Pools P) {
    pdl_enter();
    __shared__ UfSmem s_tile[WIDE_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    UfSmem& TS = s_tile[w];
    const int nw = P.g->n_wide;
    for (int k = blockIdx.x * WIDE_WARPS + w; k < nw; k += gridDim.x * WIDE_WARPS) {
        const int pid = P.wide[k];
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const int q = P.p_q[pid];
        const int yq = q / D.Lx, xq = q - yq * D.Lx;
        const int x0 = (xq / TW) * TW, y0 = (yq / TH) * TH;
        const int r = P.p_parent[pid];
        const int qr = P.p_q[r];
        const int yr = qr / D.Lx, xr = qr - yr * D.Lx;
        const unsigned long long m = load_row_mask(P.fgbits[P.st[inst].slot ^ 1], D, x0, y0);
        TS.m[lane] = m;
        warp_runs_uf(TS, m, D.conn8 != 0);
        const unsigned long long Sq = run_starts(TS.m[yq - y0]);
        const int lq = (yq - y0) * 32 + run_index(Sq, xq - x0);
        const unsigned long long S = run_starts(m);
        long long n = 0, sx = 0, sy = 0;
        unsigned long long t = S;
        int j = 0;
        const long long dy = wrap_ll((y0 + lane) - yr, D.Ly);
        while (t) {
            const int c = __ffsll(t) - 1;
            t &= t - 1;
            if (TS.par[SW(lane * 32 + j)] == lq) {
                const int len = run_length(m, c);
                for (int i = 0; i < len; ++i) sx += wrap_ll((x0 + c + i) - xr, D.Lx);
                n += len;
                sy += len * dy;
            }
            ++j;
        }
        for (int o = 16; o > 0; o >>= 1) {
            n += __shfl_xor_sync(0xffffffffu, n, o);
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) {
            atomicAdd((unsigned long long*)&P.p_accn[r], (unsigned long long)n);
            atomicAdd((unsigned long long*)&P.p_accx[r], (unsigned long long)sx);
            atomicAdd((unsigned long long*)&P.p_accy[r], (unsigned long long)sy);
        }
        __syncwarp();
    }
}

// Q10 centroids of bubbles; bucket counts; clear the root bitmap for the next
// step and the match state of every now-bubble; every non-root piece takes its
// bubble id (for the run-label pass)
__global__ void k_comp_final(Pools P) {
    pdl_enter();
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        const int r = P.p_parent[pid];
        if (r != pid) {
            P.p_comp[pid] = P.p_comp[r];   // roots were ranked by k_comp_accum
            continue;
        }
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const InstState& S = P.st[inst];
        const int q = P.p_q[pid];
        const int yq = q / D.Lx, xq = q - yq * D.Lx;
        P.rootbits[D.word_off + (long long)yq * D.wpr + (xq >> 5)] = 0u;
        // root counts per group return to zero for the next step
        atomicSub(&P.rgcnt[D.grp_off + (long long)yq * D.gpr + (xq >> 5) / RGW], 1);
        const int c = P.p_comp[pid];
        if (c >= D.comp_cap) continue;
        // match state of now-bubble c, filled by the graph stage of this step
        P.best_p[D.comp_off + c] = 0ull;
        P.inv[D.comp_off + c] = -1;
        P.active[D.comp_off + c] = 0;
        const long long nn = P.p_accn[pid];
        const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
        // round half up: floor((2p + n) / 2n) with p = 1024 * S
        long long cx = (long long)Q * xq + floordiv_ll(2 * (long long)Q * P.p_accx[pid] + nn, 2 * nn);
        long long cy = (long long)Q * yq + floordiv_ll(2 * (long long)Q * P.p_accy[pid] + nn, 2 * nn);
        cx %= MX; if (cx < 0) cx += MX;
        cy %= MY; if (cy < 0) cy += MY;
        P.cq[S.slot ^ 1][D.comp_off + c] = make_int2((int)cx, (int)cy);
        const int bx = (int)(cx / Q) / S.B, by = (int)(cy / Q) / S.B;
        if (vd_in(P, CHK_BUCKET, (long long)by * S.nbx + bx, (long long)S.nbx * S.nby))
            atomicAdd(&P.bcnt[D.bucket_off + (long long)by * S.nbx + bx], 1);
    }
}

// counting-sort scatter of centroids into bucket order (counts return to zero)
__global__ void k_bucket_scatter(Pools P) {
    pdl_enter();
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        if (P.p_parent[pid] != pid) continue;
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const InstState& S = P.st[inst];
        const int c = P.p_comp[pid];
        if (c >= D.comp_cap) continue;
        const int now = S.slot ^ 1;
        const int2 v = P.cq[now][D.comp_off + c];
        const long long bk = (long long)((v.y / Q) / S.B) * S.nbx + (v.x / Q) / S.B;
        if (!vd_in(P, CHK_BUCKET, bk, (long long)S.nbx * S.nby)) continue;
        const int pos = P.boff[now][D.bucket_off + bk] + atomicSub(&P.bcnt[D.bucket_off + bk], 1) - 1;
        if (!vd_in(P, CHK_BUCKET, pos, D.comp_cap)) continue;
        P.bcq[now][D.comp_off + pos] = v;
        P.bid[now][D.comp_off + pos] = c;
    }
}

// ---------------------------------------------------------------------------
// Label pass: final labels from the stored bits; overlap histogram with the
// previous frame's labels (Section 3.2.3)
// ---------------------------------------------------------------------------
constexpr int LBL_WARPS = 4;    // tiles per block in the label pass
constexpr int WSET = 64;        // per-warp overlap set (power of two)

// ---------------------------------------------------------------------------
// Run labels and the overlap histogram (Sections 3.1 and 3.2.3), one warp per
// 64 x 32 labelling tile, lane r on tile row r. Every run of the frame gets
// the bubble label of its piece (kept per slot for the next frame and for
// label queries). The sites shared by bubble i of the past frame and bubble j
// now form, in each row, runs of (past mask AND now mask); each such run lies
// inside one past run and one now run, so the overlap histogram is a sum of
// run lengths over (past label, now label) pairs and no site is visited.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(32 * LBL_WARPS, 10) void k_run_labels(Pools P, StepTable T) {
    pdl_enter();
    __shared__ int s_lab[LBL_WARPS][RUNS];
    __shared__ unsigned long long s_key[LBL_WARPS][WSET];
    __shared__ unsigned s_cnt[LBL_WARPS][WSET];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * LBL_WARPS + w;
    if (b >= T.tileA_pre[T.n_act]) return;
    const int a = warp_seg_of_int(T.tileA_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileA_pre[a];
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const int now = S.slot ^ 1;
    int* lab = s_lab[w];
    unsigned long long* skey = s_key[w];
    unsigned* scnt = s_cnt[w];

    // 1. bubble label of each run of this row
    const unsigned long long m = load_row_mask(P.fgbits[now], D, x0, y0);
    const unsigned long long Sn = run_starts(m);
    const int nr = __popcll(Sn);
    const int rrow = run_row_base(nr);
    const long long rbase = (long long)(D.tile_off + t) * RUNS + rrow;
    for (int j0 = 0; j0 < nr; j0 += 4) {   // four runs' loads in flight at once
        int pid[4], l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pid[k] = j0 + k < nr ? P.rp[rbase + j0 + k] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            l[k] = (pid[k] >= 0 && vd_in(P, CHK_RUN_LABEL, pid[k], P.piece_cap)) ? P.p_comp[pid[k]] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (j0 + k < nr && vd_in(P, CHK_RUN_LABEL, rrow + j0 + k, RUNS)) {
                P.rl[now][rbase + j0 + k] = l[k];
                lab[SW(lane * 32 + j0 + k)] = l[k];
            }
    }
    if (!S.has_prev || D.match_rule) return;   // warp-uniform; the centroid match needs no overlaps

    // 2. overlap runs with the past frame (same lattice, same tile)
    for (int k = lane; k < WSET; k += 32) {
        skey[k] = EMPTY_KEY;
        scnt[k] = 0;
    }
    __syncwarp();
    const int pb = S.prev_buf;
    const bool same = S.prev_same != 0;   // past frame labelled in this step: its runs still hold piece ids
    const InstDesc& DP = P.desc[S.prev_inst];
    const unsigned long long mp = load_row_mask(P.fgbits[pb], DP, x0, y0);
    const unsigned long long Sp = run_starts(mp);
    const long long pbase = (long long)(DP.tile_off + t) * RUNS + run_row_base(__popcll(Sp));
    const unsigned long long A = m & mp;
    unsigned long long As = run_starts(A);
    const int nA = __reduce_max_sync(0xffffffffu, __popcll(As));
    for (int i0 = 0; i0 < nA; i0 += 4) {   // all lanes: the set insertion is warp-wide
        // four overlap runs at a time: their past-label loads are in flight together
        unsigned len[4];
        int ln[4], lp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            len[k] = 0;
            ln[k] = -1;
            lp[k] = -1;
            if (As) {
                const int c = __ffsll(As) - 1;
                As &= As - 1;
                len[k] = run_length(A, c);
                ln[k] = lab[SW(lane * 32 + run_index(Sn, c))];
                const int jp = run_index(Sp, c);
                lp[k] = same ? P.rp[pbase + jp] : P.rl[pb][pbase + jp];
            }
        }
        if (same) {   // the past frame's runs hold piece ids: one more step to labels
#pragma unroll
            for (int k = 0; k < 4; ++k) lp[k] = lp[k] >= 0 ? P.p_comp[lp[k]] : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned long long key =
                (ln[k] >= 0 && lp[k] >= 0) ? (((unsigned long long)(unsigned)lp[k] << 32) | (unsigned)ln[k]) : EMPTY_KEY;
            unsigned csum = 0;
            if (!warp_set_add(skey, scnt, WSET, key, len[k], &csum)) ovl_global_insert(P, D, inst, key, csum);
        }
    }
    __syncwarp();
    // append the tile's (past, now, count) triples (one reservation per round);
    // k_merge_lists adds them into the overlap hash
    for (int kb = 0; kb < WSET; kb += 32) {
        const unsigned long long key = skey[kb + lane];
        const bool has = key != EMPTY_KEY;
        const unsigned mk = __ballot_sync(0xffffffffu, has);
        if (!mk) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(&P.st[inst].n_oapp, __popc(mk));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (has) {
            const int pos = base + __popc(mk & ((1u << lane) - 1u));
            if (pos < D.ovl_cap && vd_in(P, CHK_OVL_APPEND, pos, D.ovl_cap)) {
                P.oapp_key[D.ovl_off + pos] = key;
                P.oapp_cnt[D.ovl_off + pos] = scnt[kb + lane];
            } else {
                ovl_global_insert(P, D, inst, key, scnt[kb + lane]);   // list full: insert directly
            }
        }
    }
}

// per-site labels of one instance's frame in `slot`, from its foreground bits
// and run labels (-1 for background)
// per-site labels of one instance's frame in `slot` from its run labels: one
// warp per labelling tile, lane r takes row r's mask and run base, then the
// warp writes the tile row by row (lanes on columns)
constexpr int EXP_WARPS = 8;
__global__ __launch_bounds__(32 * EXP_WARPS) void k_expand_labels(Pools P, int inst, int slot, int* out) {
    const InstDesc& D = P.desc[inst];
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * EXP_WARPS + (threadIdx.x >> 5);
    if (t >= D.ntx * D.nty) return;
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const int ncols = min(TW, D.Lx - x0), nrows = min(TH, D.Ly - y0);
    const unsigned long long m = load_row_mask(P.fgbits[slot], D, x0, y0);
    const int rrow = run_row_base(__popcll(run_starts(m)));
    const int* rl = P.rl[slot] + (long long)(D.tile_off + t) * RUNS;
    for (int r = 0; r < nrows; ++r) {
        const unsigned long long mr = __shfl_sync(0xffffffffu, m, r);
        const int br = __shfl_sync(0xffffffffu, rrow, r);
        const unsigned long long Sr = run_starts(mr);
        int* row = out + (long long)(y0 + r) * D.Lx + x0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            if (c < ncols) row[c] = ((mr >> c) & 1ull) ? rl[br + run_index(Sr, c)] : -1;
        }
    }
}

void launch_expand_labels(cudaStream_t s, const Pools& P, int inst, int slot, int* out, int n_tiles) {
    k_expand_labels<<<(n_tiles + EXP_WARPS - 1) / EXP_WARPS, 32 * EXP_WARPS, 0, s>>>(P, inst, slot, out);
}

void launch_ccl_tiles(const Launch& L) {
    launch_step(L, k_threshold, dim3((L.total_tilesA + THR_WARPS - 1) / THR_WARPS), dim3(32 * THR_WARPS), L.P, L.T);
    launch_step(L, k_ccl_tiles, dim3((L.total_tilesA + CCL_WARPS - 1) / CCL_WARPS), dim3(32 * CCL_WARPS), L.P, L.T);
}

void launch_ccl_rest(const Launch& L) {
    if (L.total_tilesA > 0)
        launch_step(L, k_ccl_merge, dim3((L.total_tilesA + MERGE_WARPS - 1) / MERGE_WARPS), dim3(32 * MERGE_WARPS), L.P,
                    L.T);
    launch_step(L, k_ccl_flatten, dim3(L.grid_wide), dim3(256), L.P);
    launch_plan(L, 1, ends_bit(SCAN_BUCKETS));
    launch_scan(L, SCAN_ROOTBITS);
    launch_step(L, k_comp_accum, dim3(L.grid_wide), dim3(256), L.P);
    launch_step(L, k_comp_wide, dim3(L.grid_items), dim3(32 * WIDE_WARPS), L.P);
    launch_step(L, k_comp_final, dim3(L.grid_wide), dim3(256), L.P);
    launch_scan(L, SCAN_BUCKETS);
    launch_step(L, k_bucket_scatter, dim3(L.grid_wide), dim3(256), L.P);
}

void launch_labels(const Launch& L) {
    launch_step(L, k_run_labels, dim3((L.total_tilesA + LBL_WARPS - 1) / LBL_WARPS), dim3(32 * LBL_WARPS), L.P, L.T);
}

}  // namespace vd
