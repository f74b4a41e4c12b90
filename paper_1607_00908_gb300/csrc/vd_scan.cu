// Per-step planning and the segmented exclusive scan of libvd.
//
// A "virtual concatenation" lists, for every instance active in the step, a
// segment of items (bitmask words, buckets, bubbles). k_plan recomputes the
// segment prefixes from the per-instance counters produced by the previous
// kernels (and the end values of the offset arrays scanned next); k_scan then
// runs one single-pass scan (decoupled look-back, tiles
// claimed in order through an atomic ticket) over the whole concatenation and
// writes each item's exclusive prefix *within its own instance*: the global
// prefix minus the sum of the totals of the earlier instances, which the
// producers counted exactly.
#include "vd_internal.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// k_plan: prefixes over the active instances; bucket grid of each instance
// ---------------------------------------------------------------------------
constexpr int PLAN_THREADS = 256;

__global__ __launch_bounds__(PLAN_THREADS) void k_plan(Pools P, StepTable T, int with_comp, int ends, int pre_mask) {
    pdl_enter();
    // one block: thread per instance, block scans for the prefixes (warp
    // scans by shuffles, then the warp totals)
    __shared__ long long s_w[NPRE][PLAN_THREADS / 32];
    __shared__ long long s_carry[NPRE];
    const int n = T.n_act;
    const int tid = threadIdx.x;
    if (tid < NPRE) s_carry[tid] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += PLAN_THREADS) {
        const int a = base + tid;
        long long v[NPRE];
        for (int k = 0; k < NPRE; ++k) v[k] = 0;
        if (a < n) {
            const int inst = T.act[a];
            InstState& S = P.st[inst];
            const InstDesc& D = P.desc[inst];
            if (with_comp) {
                int K = S.K;
                S.K_roots = K;   // every root is ranked, also past the capacity
                if (K > D.comp_cap) {
                    S.err |= ERR_COMP_CAP;
                    K = D.comp_cap;
                    S.K = K;
                }
                if (K > 0) {
                    // bucket side ~ a tuned fraction of the mean spacing of centres,
                    // clamped to [4, 64] sites
                    const double sp = sqrt((double)D.Lx * (double)D.Ly / (double)K) * (0.01 * D.bucket_pct);
                    int B = (int)(sp + 0.5);
                    B = B < 4 ? 4 : (B > 64 ? 64 : B);
                    S.B = B;
                    S.nbx = (D.Lx + B - 1) / B;
                    S.nby = (D.Ly + B - 1) / B;
                } else {
                    S.B = 4; S.nbx = 0; S.nby = 0;
                }
                const int nw = S.slot ^ 1;   // the grid is kept with the frame's buffer
                S.Bs[nw] = S.B;
                S.nbxs[nw] = S.nbx;
                S.nbys[nw] = S.nby;
                if (S.prev_same) {
                    // the past frame was labelled in this step by instance prev_inst
                    const int kp = P.st[S.prev_inst].K;
                    const int cap = P.desc[S.prev_inst].comp_cap;
                    S.K_prev = kp < cap ? kp : cap;
                }
            }
            const int K = S.K < D.comp_cap ? S.K : D.comp_cap;
            v[PRE_K] = K;
            v[PRE_KP] = S.has_prev ? S.K_prev : 0;
            v[PRE_NB] = K > 0 ? (long long)S.nbx * S.nby : 0;
            v[PRE_E] = S.n_edge_list;
            v[PRE_EP] = S.has_prev ? S.E_prev : 0;
            v[PRE_O] = S.n_ovl < D.ovl_cap ? S.n_ovl : D.ovl_cap;
            v[PRE_FB] = S.n_break;
            v[PRE_FA] = S.n_arise;
            v[PRE_EA] = S.n_eapp < D.edge_cap ? S.n_eapp : D.edge_cap;
            v[PRE_OA] = S.n_oapp < D.ovl_cap ? S.n_oapp : D.ovl_cap;
            v[PRE_KR] = S.K_roots;
            // end values of the offset arrays (off[size] = total) of the scans that follow
            const int now = S.slot ^ 1;
            if (ends & ends_bit(SCAN_BUCKETS)) P.boff[now][D.bucket_off + (long long)S.nbx * S.nby] = S.K;
            if (ends & ends_bit(SCAN_DEG)) P.rowoff[now][D.comp_off + S.K] = 2 * S.n_edge_list;
            if (ends & ends_bit(SCAN_FLIPS)) P.foff[D.comp_off + S.K] = S.n_break;
            if (ends & ends_bit(SCAN_FLIPS_A)) P.foff_a[D.comp_off + S.K] = S.n_arise;
        }
        const int lane = tid & 31, wid = tid >> 5;
        long long inc[NPRE];
#pragma unroll
        for (int k = 0; k < NPRE; ++k) {
            long long x = v[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            inc[k] = x;
            if (lane == 31) s_w[k][wid] = x;
        }
        __syncthreads();
        if (a < n)
            for (int k = 0; k < NPRE; ++k) {
                long long before = s_carry[k];
                for (int w = 0; w < wid; ++w) before += s_w[k][w];
                if (pre_mask & pre_bit(k)) pre_arr(T, k)[a] = before + inc[k] - v[k];
            }
        __syncthreads();
        if (tid < NPRE)
            for (int w = 0; w < PLAN_THREADS / 32; ++w) s_carry[tid] += s_w[tid][w];
        __syncthreads();
    }
    if (tid < NPRE && (pre_mask & pre_bit(tid))) pre_arr(T, tid)[n] = s_carry[tid];
}

// ---------------------------------------------------------------------------
// k_scan
// ---------------------------------------------------------------------------
struct ScanSel {
    int seg;      // PreIdx of segment sizes, or -1 for root groups (static table)
    int base;     // PreIdx of output totals
    int mul;      // an instance's total is mul x its entry in base
};

__device__ __forceinline__ ScanSel scan_sel(int kind) {
    switch (kind) {
        case SCAN_ROOTBITS: return {-1, PRE_KR, 1};   // ranks count every root, clamped or not
        case SCAN_BUCKETS: return {PRE_NB, PRE_K, 1};
        case SCAN_DEG: return {PRE_K, PRE_E, 2};      // every link is in the rows of both ends
        case SCAN_FLIPS: return {PRE_K, PRE_FB, 1};
        default: return {PRE_K, PRE_FA, 1};
    }
}

__device__ __forceinline__ int scan_value(const Pools& P, int kind, int inst, long long j) {
    const InstDesc& D = P.desc[inst];
    switch (kind) {
        case SCAN_ROOTBITS: return P.rgcnt[D.grp_off + j];
        case SCAN_BUCKETS: return P.bcnt[D.bucket_off + j];
        case SCAN_DEG: return P.deg[D.comp_off + j];
        case SCAN_FLIPS: return P.fcnt[D.comp_off + j];
        default: return P.fcnt_a[D.comp_off + j];
    }
}

__device__ __forceinline__ void scan_write(const Pools& P, int kind, int inst, long long j, int v) {
    const InstDesc& D = P.desc[inst];
    switch (kind) {
        case SCAN_ROOTBITS:
            // the counts stay (a tile whose wait gives up re-reads them);
            // k_comp_final returns them to zero
            P.rankpre[D.grp_off + j] = v;
            break;
        case SCAN_BUCKETS: P.boff[P.st[inst].slot ^ 1][D.bucket_off + j] = v; break;
        case SCAN_DEG: P.rowoff[P.st[inst].slot ^ 1][D.comp_off + j] = v; break;
        case SCAN_FLIPS: P.foff[D.comp_off + j] = v; break;
        default: P.foff_a[D.comp_off + j] = v; break;
    }
}

constexpr unsigned ST_AGG = 1u, ST_INC = 2u;
constexpr int SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ void publish(unsigned long long* f, unsigned epoch, unsigned st, int v) {
    unsigned long long w = ((unsigned long long)epoch << 34) | ((unsigned long long)st << 32) | (unsigned)v;
    __threadfence();
    *(volatile unsigned long long*)f = w;
}

// kind2 >= 0: a second scan over the same segments in the same launch (tiles
// numbered after the first scan's); each scan keeps its own flags and tag
__global__ __launch_bounds__(SCAN_THREADS) void k_scan(Pools P, StepTable T, int kind1, int kind2) {
    pdl_enter();
    __shared__ int s_tile;
    __shared__ long long s_pre[SEG_CACHE];
    __shared__ int s_act[SEG_CACHE];
    __shared__ int s_warp[SCAN_THREADS / 32];
    __shared__ long long s_excl;
    __shared__ long long s_wsum[SCAN_THREADS / 32];
    __shared__ int s_fail;
    const ScanSel sel1 = scan_sel(kind1);
    const int n = T.n_act;
    const long long* seg0 = sel1.seg < 0 ? T.grp_pre : pre_arr(T, sel1.seg);
    const long long total = seg0[n];
    const long long ntiles1 = (total + SCAN_TILE - 1) / SCAN_TILE;
    const long long ntiles = kind2 >= 0 ? 2 * ntiles1 : ntiles1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // blocks beyond the number of tiles never take a ticket
    if ((long long)blockIdx.x >= ntiles) return;
    const int* act;
    const long long* seg = seg_table(seg0, T.act, n, s_pre, s_act, &act);

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&P.g->scan_ticket[kind1], 1);
        __syncthreads();
        const long long ticket = s_tile;
        if (ticket >= ntiles) break;
        const bool second = ticket >= ntiles1;
        const int kind = second ? kind2 : kind1;
        const long long tile = second ? ticket - ntiles1 : ticket;
        if (tile >= P.scan_flag_cap) break;
        const long long start = tile * SCAN_TILE;
        const ScanSel sel = scan_sel(kind);
        const long long* base = pre_arr(T, sel.base);
        // every scan of a step has its own tag (step count, kind)
        const unsigned epoch = ((*(volatile unsigned*)&P.g->scan_step << 3) | (unsigned)kind) & 0x3FFFFFFFu;
        // test support: a tile that withholds its flag, and a shorter wait for
        // that scan only
        const bool dbg = P.g->dbg_tile != 0 && P.g->dbg_kind == kind;
        const bool hold = dbg && P.g->dbg_tile == tile + 1;
        const int spin_limit = (dbg && P.g->dbg_spin > 0) ? P.g->dbg_spin : SPIN_LIMIT;

        // load SCAN_ITEMS consecutive items per thread
        int v[SCAN_ITEMS];
        int tsum = 0;
        const long long g0 = start + (long long)threadIdx.x * SCAN_ITEMS;
        int a = -1, inst = 0;
        long long lo = 0, hi = -1;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const long long g = g0 + i;
            int x = 0;
            if (g < total) {
                if (g >= hi) {
                    a = seg_of(seg, n, g);
                    lo = seg[a];
                    hi = seg[a + 1];
                    inst = act[a];
                }
                x = scan_value(P, kind, inst, g - lo);
            }
            v[i] = x;
            tsum += x;
        }
        // block exclusive scan of thread sums
        int inc = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        int wpre = 0, btot = 0;
#pragma unroll
        for (int w = 0; w < SCAN_THREADS / 32; ++w) {
            int t = s_warp[w];
            if (w < warp) wpre += t;
            btot += t;
        }
        const int texcl = wpre + inc - tsum;

        if (warp == 0) {
            // warp-parallel decoupled look-back over windows of 32 predecessors
            // each scan kind has its own flags
            unsigned long long* flags = P.scan_flags + (long long)kind * P.scan_flag_cap;
            long long excl = 0;
            bool fail = false;
            if (tile == 0) {
                if (lane == 0 && !hold) publish(&flags[0], epoch, ST_INC, btot);
            } else {
                if (lane == 0 && !hold) publish(&flags[tile], epoch, ST_AGG, btot);
                long long top = tile - 1;
                int spins = 0;
                for (;;) {
                    const long long idx = top - lane;
                    bool ready = true, inc = true;
                    int val = 0;
                    if (idx >= 0) {
                        const unsigned long long f = *(volatile unsigned long long*)&flags[idx];
                        const unsigned fe = (unsigned)(f >> 34), fs = (unsigned)(f >> 32) & 3u;
                        ready = (fe == epoch) && fs != 0u;
                        inc = ready && fs == ST_INC;
                        val = (int)(unsigned)f;
                    }
                    const unsigned incm = __ballot_sync(0xffffffffu, inc);
                    const unsigned nrdy = __ballot_sync(0xffffffffu, !ready);
                    const int first = incm ? __ffs(incm) - 1 : 31;
                    const unsigned need = (first >= 31) ? 0xffffffffu : ((2u << first) - 1u);
                    if (nrdy & need) {
                        if (++spins > spin_limit) {   // give up: flag the error, never hang
                            if (lane == 0) atomicOr(&P.g->err, ERR_TIMEOUT);
                            fail = true;
                            break;
                        }
                        continue;
                    }
                    __threadfence();
                    const int part = __reduce_add_sync(0xffffffffu, (unsigned)((lane <= first) ? val : 0));
                    excl += part;
                    if (incm) break;
                    top -= 32;
                }
                if (lane == 0 && !hold && !fail) publish(&flags[tile], epoch, ST_INC, (int)(excl + btot));
            }
            if (lane == 0) {
                s_excl = excl;
                s_fail = fail ? 1 : 0;
            }
        }
        __syncthreads();
        if (s_fail) {
            // the wait gave up: the exclusive prefix is summed directly from
            // every earlier item (slow, only on this path), so the offsets stay
            // exact and the tiles after this one see a correct flag
            long long acc = 0;
            int fa = -1, finst = 0;
            long long flo = 0, fhi = -1;
            for (long long g = threadIdx.x; g < start; g += SCAN_THREADS) {
                if (g >= fhi || g < flo) {
                    fa = seg_of(seg, n, g);
                    flo = seg[fa];
                    fhi = seg[fa + 1];
                    finst = act[fa];
                }
                acc += scan_value(P, kind, finst, g - flo);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) s_wsum[warp] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                long long tot = 0;
                for (int k = 0; k < SCAN_THREADS / 32; ++k) tot += s_wsum[k];
                s_excl = tot;
                if (!hold)
                    publish(P.scan_flags + (long long)kind * P.scan_flag_cap + tile, epoch, ST_INC, (int)(tot + btot));
            }
            __syncthreads();
        }
        long long run = s_excl + texcl;
        a = -1; lo = 0; hi = -1;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            const long long g = g0 + i;
            if (g < total) {
                if (g >= hi) {
                    a = seg_of(seg, n, g);
                    lo = seg[a];
                    hi = seg[a + 1];
                    inst = act[a];
                }
                // after a wait that gave up, `run` may fall short of the true
                // prefix; the clamp keeps every offset inside its instance's range
                const long long w = run - sel.mul * base[a];
                if (vd_in(P, CHK_SCAN_WRITE, g - lo, hi - lo))
                    scan_write(P, kind, inst, g - lo, (int)(w > 0 ? w : 0));
                run += v[i];
            }
        }
        __syncthreads();
    }
}

void launch_plan(const Launch& L, int with_comp, int ends, int pre_mask) {
    launch_step(L, k_plan, dim3(1), dim3(PLAN_THREADS), L.P, L.T, with_comp, ends, pre_mask);
}

void launch_scan(const Launch& L, ScanKind kind) {
    launch_step(L, k_scan, dim3(L.grid_items), dim3(SCAN_THREADS), L.P, L.T, (int)kind, -1);
}

void launch_scan2(const Launch& L, ScanKind kind1, ScanKind kind2) {
    launch_step(L, k_scan, dim3(L.grid_items), dim3(SCAN_THREADS), L.P, L.T, (int)kind1, (int)kind2);
}

}  // namespace vd
