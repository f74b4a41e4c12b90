// Adjacency lists, isomorphism and topology changes (Sections 3.2.2-3.2.4).
//
// Links of a frame are kept as a CSR adjacency list of both directions: row a
// holds every label linked to a, sorted (the paper's compressed adjacency
// matrix, stored for both ends of each link). The isomorphism Phi between past
// and now labels is the mutual best overlap. For each now-bubble a with a past
// counterpart ia = Phi^-1(a), the translated past row is Phi of the past
// neighbours of ia that lie above a, sorted (the paper's "translation"; with
// both directions stored, row a needs only past row ia, so no translated CSR
// has to be counted and scattered). One thread per now row then merges the
// translated row with the now row's entries above a: entries only in the past
// row are breaking links, entries only in the now row are arising links.
// Labels outside Phi's domain or image are excluded, as the paper does for
// appearing and vanishing bubbles. Row-by-row output keeps both lists sorted
// by now-key.
#include "vd_internal.cuh"

namespace vd {

// every item of the virtual concatenation `which` (all threads of the block
// must call this: the segment table is copied to shared memory first)
template <class F>
__device__ __forceinline__ void for_items(const StepTable& T, int which, F f) {
    __shared__ long long s_pre[SEG_CACHE];
    __shared__ int s_act[SEG_CACHE];
    const int* act;
    const long long* pre = seg_table(pre_arr(T, which), T.act, T.n_act, s_pre, s_act, &act);
    const long long total = pre[T.n_act];
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int a = seg_of(pre, T.n_act, g);
        f(act[a], g - pre[a]);
    }
}

// ---------------------------------------------------------------------------
// step begin / finish
// ---------------------------------------------------------------------------
// Hash slots are returned to empty by the kernels that read the listed ones;
// a frame whose link or overlap list overflowed left keys that were never
// listed. The first kernel of the next step clears those instances' tables
// (whole block per instance; only after an overflow).
constexpr int CLEAR_LIST = 64;
__device__ void clear_overflowed_hashes(const Pools& P, const StepTable& T) {
    __shared__ int s_list[CLEAR_LIST];
    __shared__ int s_n;
    if (!*(volatile int*)&P.g->lists_over) return;   // the usual case: nothing overflowed
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < T.n_act; a += blockDim.x) {
        const int inst = T.act[a];
        if (P.st[inst].err & (ERR_EDGE_CAP | ERR_OVL_CAP)) {
            const int k = atomicAdd(&s_n, 1);
            if (k < CLEAR_LIST) s_list[k] = inst;
        }
    }
    __syncthreads();
    const int n = s_n;
    // more overflowed instances than the list holds: clear every active one
    const int m = n > CLEAR_LIST ? T.n_act : n;
    for (int i = 0; i < m; ++i) {
        const int inst = n > CLEAR_LIST ? T.act[i] : s_list[i];
        const InstDesc& D = P.desc[inst];
        const int e = P.st[inst].err;
        if (e & ERR_EDGE_CAP)
            for (long long h = threadIdx.x; h <= D.ehash_mask; h += blockDim.x) P.ehash[D.ehash_off + h] = EMPTY_KEY;
        if (e & ERR_OVL_CAP)
            for (long long h = threadIdx.x; h <= D.ohash_mask; h += blockDim.x) {
                P.ohash[D.ohash_off + h] = EMPTY_KEY;
                P.oval[D.ohash_off + h] = 0;
            }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicSub(&P.g->lists_over, n);   // the active ones among them are clean now
}

__global__ void k_step_begin(Pools P, StepTable T) {
    pdl_enter();
    clear_overflowed_hashes(P, T);   // the launch is one block
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.g->n_pieces = 0;
        P.g->n_wide = 0;
        P.g->err = 0;   // errors of the previous step stay in its instances' states
        P.g->chk_id = 0;
        P.g->chk_index = 0;
        P.g->scan_step = (P.g->scan_step + 1) & 0x07FFFFFFu;   // new tags for this step's scans
        for (int k = 0; k < 8; ++k) P.g->scan_ticket[k] = 0;
    }
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < T.n_act; a += gridDim.x * blockDim.x) {
        const int inst = T.act[a];
        InstState& S = P.st[inst];
        const InstDesc& D = P.desc[inst];
        S.field = P.fields[inst];
        S.pitch = P.pitches[inst];
        // where this step's past frame lives
        const int pi = D.seq_prev;
        const InstState& SP = P.st[pi];
        S.prev_inst = pi;
        S.prev_same = D.seq_same;
        if (D.seq_same) {
            S.prev_buf = SP.slot ^ 1;     // written by instance pi in this step
            S.has_prev = 1;
            S.K_prev = 0;                 // known after labelling (k_plan)
        } else {
            S.prev_buf = SP.slot;         // written by instance pi in an earlier step
            S.has_prev = (SP.frame > 0 && SP.last_ok) ? 1 : 0;
            S.K_prev = S.has_prev ? SP.Kb[SP.slot] : 0;
        }
        S.K = 0;
        S.E = 0;
        S.n_matched = 0;
        S.n_break = 0;
        S.n_arise = 0;
        S.n_wide = 0;
        S.n_ovl = 0;
        S.n_edge_list = 0;
        S.n_eapp = 0;
        S.n_oapp = 0;
        S.err = 0;
    }
}

// end of a step for one instance: errors, counts, the frame becomes the past
__device__ __forceinline__ void finish_instance(const Pools& P, int inst) {
    {
        InstState& S = P.st[inst];
        S.err |= P.g->err;
        // a past frame from this step that overflowed makes this frame's changes unreliable
        if (S.has_prev && S.prev_same && P.st[S.prev_inst].err) S.err |= ERR_PREV;
        const int ecap = P.desc[inst].edge_cap;
        S.E = S.n_edge_list < ecap ? S.n_edge_list : ecap;
        S.rep_K_prev = S.has_prev ? S.K_prev : 0;
        const int now = S.slot ^ 1;
        S.Kb[now] = S.K;
        S.Eb[now] = S.E;
        S.E_prev = S.E;
        S.slot = now;
        S.last_ok = S.err ? 0 : 1;
        S.frame += 1;
    }
}

__global__ void k_step_finish(Pools P, StepTable T) {
    pdl_enter();
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < T.n_act; a += gridDim.x * blockDim.x)
        finish_instance(P, T.act[a]);
}

// sorted link keys of one instance's frame in `slot`: the entries above the
// diagonal of each row, placed by a block-wide scan of their counts
constexpr int EK_THREADS = 1024;
__global__ __launch_bounds__(EK_THREADS) void k_edge_keys(Pools P, int inst, int slot, unsigned long long* out) {
    __shared__ int s_warp[EK_THREADS / 32];
    __shared__ int s_base;
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int K = min(S.Kb[slot], D.comp_cap);
    const int cap = 2 * D.edge_cap;
    const int* ro = P.rowoff[slot] + D.comp_off;
    const int* cl = P.cols[slot] + 2 * D.edge_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int a0 = 0; a0 < K; a0 += EK_THREADS) {
        const int a = a0 + threadIdx.x;
        int s = 0, e = 0;
        if (a < K) {
            s = min(ro[a], cap);
            e = max(min(ro[a + 1], cap), s);   // never a negative row length
            while (s < e && cl[s] < a) ++s;   // rows are sorted: the entries above a are a suffix
        }
        const int cnt = e - s;
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        int pre = s_base, tot = 0;
        for (int w = 0; w < EK_THREADS / 32; ++w) {
            if (w < warp) pre += s_warp[w];
            tot += s_warp[w];
        }
        int pos = pre + inc - cnt;
        for (int k = s; k < e; ++k, ++pos)
            if (pos < D.edge_cap) out[pos] = edge_key(a, cl[k]);
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
}

void launch_edge_keys(cudaStream_t s, const Pools& P, int inst, int slot, unsigned long long* out) {
    k_edge_keys<<<1, EK_THREADS, 0, s>>>(P, inst, slot, out);
}

// ---------------------------------------------------------------------------
// CSR of the now links
// ---------------------------------------------------------------------------
__device__ __forceinline__ void csr_scatter_item(const Pools& P, int inst, long long j) {
    {
        const InstDesc& D = P.desc[inst];
        if (j >= D.edge_cap) return;
        const int now = P.st[inst].slot ^ 1;
        const int slot = P.elist[D.edge_off + j];
        unsigned long long* H = P.ehash + D.ehash_off;
        const unsigned long long key = H[slot];
        H[slot] = EMPTY_KEY;
        const int lo = (int)(key >> 32), hi = (int)(key & 0xffffffffu);
        const int* ro = P.rowoff[now] + D.comp_off;
        int* cl = P.cols[now] + 2 * D.edge_off;
        const int cap = 2 * D.edge_cap;
        const int plo = ro[lo] + atomicSub(&P.deg[D.comp_off + lo], 1) - 1;
        const int phi_ = ro[hi] + atomicSub(&P.deg[D.comp_off + hi], 1) - 1;
        if (plo < cap && vd_in(P, CHK_CSR, plo, cap)) cl[plo] = hi;
        if (phi_ < cap && vd_in(P, CHK_CSR, phi_, cap)) cl[phi_] = lo;
    }
}

__global__ void k_csr_scatter(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_E, [&](int inst, long long j) { csr_scatter_item(P, inst, j); });
}

// ascending sort of a short row in place: insertion sort up to 32 entries,
// heap sort beyond (rows of very high degree stay O(d log d))
__device__ __forceinline__ void sift_down(int* v, int i, int n) {
    const int x = v[i];
    for (;;) {
        int c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && v[c + 1] > v[c]) ++c;
        if (v[c] <= x) break;
        v[i] = v[c];
        i = c;
    }
    v[i] = x;
}

__device__ void sort_row(int* v, int n) {
    if (n <= 32) {
        for (int i = 1; i < n; ++i) {
            const int x = v[i];
            int j = i - 1;
            while (j >= 0 && v[j] > x) {
                v[j + 1] = v[j];
                --j;
            }
            v[j + 1] = x;
        }
        return;
    }
    for (int i = n / 2 - 1; i >= 0; --i) sift_down(v, i, n);
    for (int e = n - 1; e > 0; --e) {
        const int t = v[0];
        v[0] = v[e];
        v[e] = t;
        sift_down(v, 0, e);
    }
}

constexpr int RLOC = 32;   // rows up to this length are handled in a local array (loads issued together)

__device__ __forceinline__ void csr_sort_item(const Pools& P, int inst, long long a) {
    const InstDesc& D = P.desc[inst];
    // the scatter returned the degree counts of the listed links to zero;
    // links past the list's capacity (an overflowed frame) were counted but
    // not listed, so the row's count is cleared here for the next step
    P.deg[D.comp_off + a] = 0;
    const int now = P.st[inst].slot ^ 1;
    const int* ro = P.rowoff[now] + D.comp_off;
    const int cap = 2 * D.edge_cap;
    const int s = min(ro[a], cap), e = min(ro[a + 1], cap);
    int* row = P.cols[now] + 2 * D.edge_off + s;
    const int n = e - s;
    if (n > RLOC) {
        sort_row(row, n);
        return;
    }
    int v[RLOC];
#pragma unroll 8
    for (int k = 0; k < n; ++k) v[k] = row[k];
    sort_row(v, n);
#pragma unroll 8
    for (int k = 0; k < n; ++k) row[k] = v[k];
}

__global__ void k_csr_sort(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_K, [&](int inst, long long a) { csr_sort_item(P, inst, a); });
}

// ---------------------------------------------------------------------------
// isomorphism Phi by mutual best overlap
// ---------------------------------------------------------------------------
// pack (count, label) so that atomicMax picks the largest count, then the smallest label
__device__ __forceinline__ unsigned long long pack_best(unsigned cnt, int label) {
    return ((unsigned long long)cnt << 32) | (0xffffffffu - (unsigned)label);
}
__device__ __forceinline__ int unpack_label(unsigned long long v) {
    return (int)(0xffffffffu - (unsigned)(v & 0xffffffffu));
}

__device__ __forceinline__ void match_best_item(const Pools& P, int inst, long long j) {
    const InstDesc& D = P.desc[inst];
    const int slot = P.olist[D.ovl_off + j];
    unsigned long long* H = P.ohash + D.ohash_off;
    unsigned* V = P.oval + D.ohash_off;
    const unsigned long long key = H[slot];
    const unsigned cnt = V[slot];
    H[slot] = EMPTY_KEY;
    V[slot] = 0;
    const int p = (int)(key >> 32), n = (int)(key & 0xffffffffu);
    if (p < 0 || n < 0 || p >= D.comp_cap || n >= D.comp_cap) return;   // only after an overflow
    if (!vd_in(P, CHK_MATCH, j, D.ovl_cap)) return;
    atomicMax(&P.best_n[D.comp_off + p], pack_best(cnt, n));
    atomicMax(&P.best_p[D.comp_off + n], pack_best(cnt, p));
}

__global__ void k_match_best(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_O, [&](int inst, long long j) { match_best_item(P, inst, j); });
}

// Centroid rule (Section 3.2.3, the kinematic comparison of the two sets of
// centres): best_n(p) = the now centre nearest to past centre p, best_p(n)
// the past centre nearest to now centre n, within the match radius; Phi is
// then the mutual choice (k_match_phi). The search runs over the other
// frame's bucket grid: every centre within R sites lies in a bucket at most
// ceil(R / B) + 1 buckets away (the ragged last bucket adds one boundary).
struct CentreGrid {
    const int2* bcq;   // centres in bucket order
    const int* bid;    // their labels
    const int* boff;   // bucket offsets (nbx * nby + 1)
    int B, nbx, nby;
};

__device__ int nearest_centre(const CentreGrid& G, int2 q, int Lx, int Ly, int radius) {
    if (G.nbx <= 0 || G.nby <= 0) return -1;
    const long long MX = (long long)Q * Lx, MY = (long long)Q * Ly;
    const long long R2 = ((long long)Q * radius) * ((long long)Q * radius);
    const int rr = (radius + G.B - 1) / G.B + 1;
    int x0 = (q.x / Q) / G.B - rr, nx = 2 * rr + 1;
    int y0 = (q.y / Q) / G.B - rr, ny = 2 * rr + 1;
    if (nx >= G.nbx) { x0 = 0; nx = G.nbx; }   // the ring covers the grid: every column once
    if (ny >= G.nby) { y0 = 0; ny = G.nby; }
    int best = -1;
    long long bd = R2;
    // smallest distance along one axis from q to the centres of a bucket
    // (an arc of the ring): 0 inside it, else the nearer end
    auto gap = [&](int bi, int qv, long long M) -> long long {
        const long long lo = (long long)bi * G.B * Q, hi = min((long long)(bi + 1) * G.B * Q, M) - 1;
        if (qv >= lo && qv <= hi) return 0;
        const long long a = wrap_ll(lo - qv, M), c = wrap_ll(hi - qv, M);
        return min(a < 0 ? -a : a, c < 0 ? -c : c);
    };
    for (int iy = 0; iy < ny; ++iy) {
        const int by = ((y0 + iy) % G.nby + G.nby) % G.nby;
        const long long gy = gap(by, q.y, MY);
        if (gy * gy > R2) continue;
        for (int ix = 0; ix < nx; ++ix) {
            const int bx = ((x0 + ix) % G.nbx + G.nbx) % G.nbx;
            const long long gx = gap(bx, q.x, MX);
            if (gx * gx + gy * gy > R2) continue;   // no centre of the bucket is within the radius
            const int b = by * G.nbx + bx;
            for (int k = G.boff[b]; k < G.boff[b + 1]; ++k) {
                const int2 c = G.bcq[k];
                const long long dx = wrap_ll((long long)c.x - q.x, MX), dy = wrap_ll((long long)c.y - q.y, MY);
                const long long d = dx * dx + dy * dy;
                const int id = G.bid[k];
                if (d < bd || (d == bd && (best < 0 || id < best))) {
                    bd = d;
                    best = id;
                }
            }
        }
    }
    return best;
}

__device__ __forceinline__ void match_kin_past_item(const Pools& P, int inst, long long p) {
    const InstDesc& D = P.desc[inst];
    if (!D.match_rule) return;
    const InstState& S = P.st[inst];
    const int now = S.slot ^ 1;
    const InstDesc& DP = P.desc[S.prev_inst];
    const CentreGrid G{P.bcq[now] + D.comp_off, P.bid[now] + D.comp_off, P.boff[now] + D.bucket_off, S.B,
                       S.nbx, S.nby};
    const int2 q = P.cq[S.prev_buf][DP.comp_off + p];
    const int n = nearest_centre(G, q, D.Lx, D.Ly, D.match_radius);
    P.best_n[D.comp_off + p] = n >= 0 ? pack_best(1u, n) : 0ull;
}

__device__ __forceinline__ void match_kin_now_item(const Pools& P, int inst, long long n) {
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    if (!D.match_rule || !S.has_prev) return;
    const int now = S.slot ^ 1, pb = S.prev_buf;
    const InstDesc& DP = P.desc[S.prev_inst];
    const InstState& SP = P.st[S.prev_inst];
    const CentreGrid G{P.bcq[pb] + DP.comp_off, P.bid[pb] + DP.comp_off, P.boff[pb] + DP.bucket_off,
                       SP.Bs[pb], SP.nbxs[pb], SP.nbys[pb]};
    const int p = nearest_centre(G, P.cq[now][D.comp_off + n], D.Lx, D.Ly, D.match_radius);
    P.best_p[D.comp_off + n] = p >= 0 ? pack_best(1u, p) : 0ull;
}

__global__ void k_match_kin(Pools P, StepTable T) {
    pdl_enter();
    // past centres: the nearest now centre
    for_items(T, PRE_KP, [&](int inst, long long p) { match_kin_past_item(P, inst, p); });
    // now centres: the nearest past centre
    for_items(T, PRE_K, [&](int inst, long long n) { match_kin_now_item(P, inst, n); });
}

__device__ __forceinline__ void match_phi_item(const Pools& P, int inst, long long p) {
    const InstDesc& D = P.desc[inst];
    const unsigned long long v = P.best_n[D.comp_off + p];
    P.best_n[D.comp_off + p] = 0ull;   // zero again for the next step
    int res = -1;
    if (v != 0ull) {
        const int n = unpack_label(v);
        const unsigned long long w = P.best_p[D.comp_off + n];
        if (w != 0ull && unpack_label(w) == (int)p) {
            res = n;
            P.inv[D.comp_off + n] = (int)p;
            warp_add(&P.st[inst].n_matched, 1);
        }
    }
    P.phi[D.comp_off + p] = res;
}

__global__ void k_match_phi(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_KP, [&](int inst, long long p) { match_phi_item(P, inst, p); });
}

// ---------------------------------------------------------------------------
// translation and row comparison: breaking = translated past only, arising =
// now only
// ---------------------------------------------------------------------------
// Translated past row of now-bubble a (ia = Phi^-1(a) >= 0): Phi(b) for the
// past neighbours b of ia with Phi(b) > a, sorted, written at the past row's
// position in tcols; returns its length
__device__ int translate_row(const Pools& P, const InstDesc& D, const InstState& S, int a, int ia) {
    const InstDesc& DP = P.desc[S.prev_inst];
    const int pcap = 2 * DP.edge_cap, cap = 2 * D.edge_cap;
    const int* pro = P.rowoff[S.prev_buf] + DP.comp_off;
    const int* pcl = P.cols[S.prev_buf] + 2 * DP.edge_off;
    const int s = min(pro[ia], pcap), e = min(min(pro[ia + 1], pcap), cap);
    if (s >= e) return 0;
    int* tr = P.tcols + 2 * D.edge_off + s;
    const int* phi = P.phi + D.comp_off;
    const int n = e - s;
    int t = 0;
    if (n <= RLOC) {
        int v[RLOC];
#pragma unroll 8
        for (int k = 0; k < n; ++k) v[k] = pcl[s + k];
#pragma unroll 8
        for (int k = 0; k < n; ++k) {
            const int b = v[k];
            v[k] = (b >= 0 && b < D.comp_cap) ? phi[b] : -1;   // out of range only after an overflow
        }
        for (int k = 0; k < n; ++k)
            if (v[k] > a) v[t++] = v[k];
        sort_row(v, t);
#pragma unroll 8
        for (int k = 0; k < t; ++k) tr[k] = v[k];
    } else {
        for (int k = s; k < e; ++k) {
            const int b = pcl[k];
            if (b < 0 || b >= D.comp_cap) continue;
            const int pb = phi[b];
            if (pb > a) tr[t++] = pb;
        }
        sort_row(tr, t);
    }
    return t;
}

// Merge of the translated row tr[0..nt) with the now row's candidates: the
// entries nowv(i), i < nn, for which skip(i) is false (above a, other end
// matched), ascending
template <bool WRITE, class NowV, class Skip>
__device__ __forceinline__ void merge_row(const Pools& P, const InstDesc& D, int a, int ia, const int* tr, int nt,
                                          int nn, NowV nowv, Skip skip, int ob, int oa, int& nb, int& na) {
    const long long co = D.comp_off;
    int i = 0, j = 0;
    for (;;) {
        while (i < nn && skip(i)) ++i;
        const bool hn = i < nn, ht = j < nt;
        if (!hn && !ht) break;
        const int vn = hn ? nowv(i) : INT_MAX, vt = ht ? tr[j] : INT_MAX;
        if (vn == vt) {
            ++i;
            ++j;
        } else if (vt < vn) {   // only in the past: breaking
            if (WRITE && vd_in(P, CHK_FLIPS, ob + nb, D.edge_cap)) {
                const long long o = D.edge_off + ob + nb;
                P.brk[o] = edge_key(a, vt);
                P.brk_prev[o] = edge_key(ia, P.inv[co + vt]);
                P.active[co + a] = 1;
                P.active[co + vt] = 1;
            }
            ++nb;
            ++j;
        } else {                // only now: arising
            if (WRITE && vd_in(P, CHK_FLIPS, oa + na, D.edge_cap)) {
                P.ari[D.edge_off + oa + na] = edge_key(a, vn);
                P.active[co + a] = 1;
                P.active[co + vn] = 1;
            }
            ++na;
            ++i;
        }
    }
}

template <bool WRITE>
__device__ __forceinline__ void compare_row(const Pools& P, int inst, int a) {
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int now = S.slot ^ 1;
    const long long co = D.comp_off;
    int nb = 0, na = 0;
    int ob = 0, oa = 0;
    if (WRITE) {
        ob = P.foff[co + a];
        oa = P.foff_a[co + a];
    }
    const int ia = S.has_prev ? P.inv[co + a] : -1;
    if (ia >= 0) {
        int nt;
        const int* tr;
        {
            const InstDesc& DP = P.desc[S.prev_inst];
            const int s = min(P.rowoff[S.prev_buf][DP.comp_off + ia], 2 * DP.edge_cap);
            tr = P.tcols + 2 * D.edge_off + s;
        }
        if (WRITE) {
            nt = P.tlen[co + a];
        } else {
            nt = translate_row(P, D, S, a, ia);
            P.tlen[co + a] = nt;
        }
        const int cap = 2 * D.edge_cap;
        const int* nr = P.cols[now] + 2 * D.edge_off;
        const int s = min(P.rowoff[now][co + a], cap);
        const int n = min(P.rowoff[now][co + a + 1], cap) - s;
        if (n <= RLOC && nt <= RLOC) {
            // both rows in local arrays: loads issued together, then the merge
            int v[RLOC], w[RLOC], t[RLOC];
#pragma unroll 8
            for (int k = 0; k < n; ++k) v[k] = nr[s + k];
#pragma unroll 8
            for (int k = 0; k < n; ++k) {
                const int c = v[k];
                w[k] = (c > a && c < D.comp_cap) ? P.inv[co + c] : -1;
            }
#pragma unroll 8
            for (int k = 0; k < nt; ++k) t[k] = tr[k];
            merge_row<WRITE>(P, D, a, ia, t, nt, n, [&](int i) { return v[i]; }, [&](int i) { return w[i] < 0; },
                             ob, oa, nb, na);
        } else {
            merge_row<WRITE>(P, D, a, ia, tr, nt, n, [&](int i) { return nr[s + i]; },
                             [&](int i) {
                                 const int c = nr[s + i];
                                 return c <= a || c >= D.comp_cap || P.inv[co + c] < 0;
                             },
                             ob, oa, nb, na);
        }
    }
    if (!WRITE) {
        P.fcnt[co + a] = nb;
        P.fcnt_a[co + a] = na;
        warp_add(&P.st[inst].n_break, nb);
        warp_add(&P.st[inst].n_arise, na);
    }
}

__global__ void k_flip_count(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_K, [&](int inst, long long a) { compare_row<false>(P, inst, (int)a); });
}

__global__ void k_flip_write(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_K, [&](int inst, long long a) { compare_row<true>(P, inst, (int)a); });
}

// ---------------------------------------------------------------------------
// Event classes of the active labels (Section 3.2.4, "Extracting Topology
// Change Events"). For each active now-bubble a (its past label ia = Phi^-1(a)
// exists: flips join matched labels only):
//   c_N = active now neighbours of a, c_P = past neighbours q of ia whose
//   Phi(q) is active; bulk event point: max(c_N, c_P) >= 3;
//   boundary point of a triangulation: an end of a link whose ends share
//   exactly one neighbour; boundary event point: a boundary point of the past
//   or the now triangulation linked there to an active boundary point.
// The classes are OR-ed into the active flags above bit 0. One thread per
// active row; a row and its neighbours' rows are held in registers (up to
// DREG entries each) so that their loads are issued together, and longer
// rows are merged from global memory.
// ---------------------------------------------------------------------------
struct Graph {
    const int* ro;     // row offsets (per-instance values)
    const int* cl;     // columns
    int cap;           // columns available
    int K;             // rows
};

__device__ __forceinline__ void row_of(const Graph& G, int u, int& s, int& e) {
    s = min(G.ro[u], G.cap);
    e = min(G.ro[u + 1], G.cap);
    if (e < s) e = s;
}

// labels in both sorted lists x[0..nx) and y[0..ny), counting stops at 2
__device__ __forceinline__ int shared2(const int* x, int nx, const int* y, int ny) {
    int i = 0, j = 0, n = 0;
    while (i < nx && j < ny && n < 2) {
        const int p = x[i], q = y[j];
        n += (p == q) ? 1 : 0;
        i += (p <= q) ? 1 : 0;
        j += (q <= p) ? 1 : 0;
    }
    return n;
}

// true when one of row u's links shares exactly one neighbour
__device__ bool boundary_pt_global(const Graph& G, int u) {
    int s, e;
    row_of(G, u, s, e);
    for (int k = s; k < e; ++k) {
        const int v = G.cl[k];
        if (v < 0 || v >= G.K) continue;
        int vs, ve;
        row_of(G, v, vs, ve);
        if (shared2(G.cl + s, e - s, G.cl + vs, ve - vs) == 1) return true;
    }
    return false;
}

// The same with row u and its neighbours' rows in registers when every one
// of them has at most DREG entries (the usual Voronoi degrees): row u, the
// neighbours' row ranges and all their entries are three rounds of
// independent loads, and the shared neighbours are counted by comparisons.
constexpr int DREG = 10;

__device__ bool boundary_pt(const Graph& G, int u) {
    int s, e;
    row_of(G, u, s, e);
    const int nu = e - s;
    if (nu > DREG) return boundary_pt_global(G, u);
    int ru[DREG], vs[DREG], vn[DREG];
    bool small = true;
#pragma unroll
    for (int k = 0; k < DREG; ++k) ru[k] = k < nu ? G.cl[s + k] : -1;
#pragma unroll
    for (int k = 0; k < DREG; ++k) {
        vs[k] = 0;
        vn[k] = 0;
        const int v = ru[k];
        if (v >= 0 && v < G.K) {
            int a, b;
            row_of(G, v, a, b);
            vs[k] = a;
            vn[k] = b - a;
            small = small && (b - a) <= DREG;
        }
    }
    if (!small) return boundary_pt_global(G, u);
    bool hit = false;
#pragma unroll
    for (int k = 0; k < DREG; ++k) {
        int n = 0;
#pragma unroll
        for (int t = 0; t < DREG; ++t) {
            const int w = t < vn[k] ? G.cl[vs[k] + t] : -2;
#pragma unroll
            for (int j = 0; j < DREG; ++j) n += (ru[j] == w) ? 1 : 0;
        }
        hit = hit || (vn[k] > 0 && n == 1);
    }
    return hit;
}

__device__ __forceinline__ void events_item(const Pools& P, int inst, long long a_) {
    const int a = (int)a_;
    const InstDesc& D = P.desc[inst];
    const long long co = D.comp_off;
    if (!D.events || !(P.active[co + a] & EV_ACTIVE)) return;
    const InstState& S = P.st[inst];
    const int ia = S.has_prev ? P.inv[co + a] : -1;
    const int now = S.slot ^ 1;
    const int K = min(S.K, D.comp_cap);
    const Graph GN{P.rowoff[now] + co, P.cols[now] + 2 * D.edge_off, 2 * D.edge_cap, K};
    const int* phi = P.phi + co;
    const unsigned char* act = P.active + co;
    auto active_now = [&](int n) { return n >= 0 && n < K && (act[n] & EV_ACTIVE); };
    unsigned f = 0;
    // the now triangulation
    int c_now = 0;
    bool bnow = false, evnow = false;
    {
        int s, e;
        row_of(GN, a, s, e);
#pragma unroll 8
        for (int k = s; k < e; ++k) c_now += active_now(GN.cl[k]) ? 1 : 0;
        bnow = boundary_pt(GN, a);
        if (bnow)
            for (int k = s; k < e && !evnow; ++k) {
                const int b = GN.cl[k];
                evnow = active_now(b) && boundary_pt(GN, b);
            }
    }
    // the past triangulation, seen through Phi
    int c_past = 0;
    bool bpast = false, evpast = false;
    if (ia >= 0) {
        const InstDesc& DP = P.desc[S.prev_inst];
        const int Kp = S.K_prev;
        const Graph GP{P.rowoff[S.prev_buf] + DP.comp_off, P.cols[S.prev_buf] + 2 * DP.edge_off,
                       2 * DP.edge_cap, Kp};
        auto active_past = [&](int q) { return q >= 0 && q < Kp && q < D.comp_cap && active_now(phi[q]); };
        int s, e;
        row_of(GP, ia, s, e);
#pragma unroll 8
        for (int k = s; k < e; ++k) c_past += active_past(GP.cl[k]) ? 1 : 0;
        bpast = boundary_pt(GP, ia);
        if (bpast)
            for (int k = s; k < e && !evpast; ++k) {
                const int q = GP.cl[k];
                evpast = active_past(q) && boundary_pt(GP, q);
            }
    }
    if (max(c_now, c_past) >= 3) f |= EV_BULK;
    if (evnow || evpast) f |= EV_BOUNDARY;
    if (bnow) f |= EV_BPOINT_NOW;
    if (bpast) f |= EV_BPOINT_PAST;
    if (f) P.active[co + a] = (unsigned char)(EV_ACTIVE | f);
}

__global__ void k_events(Pools P, StepTable T) {
    pdl_enter();
    for_items(T, PRE_K, [&](int inst, long long a_) { events_item(P, inst, a_); });
}

// ---------------------------------------------------------------------------
// The graph stage with one block per instance. For batches of small lattices
// the stage above is a chain of about a dozen grid-wide launches whose items
// (rows, links, pairs) number a few thousand per instance: each launch costs
// a few dependent L2 round trips plus a kernel boundary. Here one block of
// GI_THREADS threads takes every phase of one instance, with block barriers
// between the phases: k_graph_inst_a builds the now-frame CSR and the match,
// k_graph_inst_b (after it, since a frame sequence translates the CSR the
// previous instance built in this step) counts, places and writes the flips,
// classifies the events and ends the instance's step. The per-item work is
// the same code as the grid-wide kernels; the scans are block scans over the
// instance's rows. No block waits on another.
// ---------------------------------------------------------------------------
constexpr int GI_THREADS = 1024;

template <class F>
__device__ __forceinline__ void block_items(long long n, F f) {
    for (long long j = threadIdx.x; j < n; j += blockDim.x) f(j);
}

// exclusive prefix of v(j), j < n, over the block in chunks of its size (the
// carry held in shared memory); w(j, prefix) stores each prefix. Ends with a
// barrier.
template <class V, class W>
__device__ void block_scan(int n, V v, W w) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int j = base + tid;
        const int x = j < n ? v(j) : 0;
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int t = lane < nw ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) s_warp[lane] = t;   // inclusive over warps
        }
        __syncthreads();
        if (j < n) w(j, s_carry + (wid > 0 ? s_warp[wid - 1] : 0) + inc - x);
        __syncthreads();
        if (tid == 0) s_carry += s_warp[nw - 1];
        __syncthreads();
    }
}

__global__ __launch_bounds__(GI_THREADS) void k_graph_inst_a(Pools P, StepTable T) {
    pdl_enter();
    const int inst = T.act[blockIdx.x];
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int K = min(S.K, D.comp_cap);
    const int now = S.slot ^ 1;
    const int nE = S.n_edge_list;
    const int KP = S.has_prev ? S.K_prev : 0;
    const int nO = min(S.n_ovl, D.ovl_cap);
    int* ro = P.rowoff[now] + D.comp_off;
    // CSR of the now links: row offsets = prefix of the degrees (every link
    // lies in the rows of both ends)
    if (threadIdx.x == 0) ro[K] = 2 * nE;
    block_scan(K, [&](int j) { return P.deg[D.comp_off + j]; },
               [&](int j, int pre) { if (vd_in(P, CHK_SCAN_WRITE, j, K)) ro[j] = pre; });
    block_items(nE, [&](long long j) { csr_scatter_item(P, inst, j); });
    __syncthreads();
    block_items(K, [&](long long a) { csr_sort_item(P, inst, a); });
    // the match (Section 3.2.3)
    if (D.match_rule) {
        block_items(KP, [&](long long p) { match_kin_past_item(P, inst, p); });
        block_items(K, [&](long long n) { match_kin_now_item(P, inst, n); });
    }
    __syncthreads();
    block_items(nO, [&](long long j) { match_best_item(P, inst, j); });
    __syncthreads();
    block_items(KP, [&](long long p) { match_phi_item(P, inst, p); });
}

__global__ __launch_bounds__(GI_THREADS) void k_graph_inst_b(Pools P, StepTable T) {
    pdl_enter();
    const int inst = T.act[blockIdx.x];
    const InstDesc& D = P.desc[inst];
    const int K = min(P.st[inst].K, D.comp_cap);
    block_items(K, [&](long long a) { compare_row<false>(P, inst, (int)a); });
    __syncthreads();
    // flip offsets: prefixes of the per-row counts, the totals at the end
    if (threadIdx.x == 0) {
        P.foff[D.comp_off + K] = *(volatile int*)&P.st[inst].n_break;
        P.foff_a[D.comp_off + K] = *(volatile int*)&P.st[inst].n_arise;
    }
    block_scan(K, [&](int j) { return P.fcnt[D.comp_off + j]; },
               [&](int j, int pre) { if (vd_in(P, CHK_SCAN_WRITE, j, K)) P.foff[D.comp_off + j] = pre; });
    block_scan(K, [&](int j) { return P.fcnt_a[D.comp_off + j]; },
               [&](int j, int pre) { if (vd_in(P, CHK_SCAN_WRITE, j, K)) P.foff_a[D.comp_off + j] = pre; });
    block_items(K, [&](long long a) { compare_row<true>(P, inst, (int)a); });
    __syncthreads();
    if (D.events) {
        block_items(K, [&](long long a) { events_item(P, inst, a); });
        __syncthreads();
    }
    if (threadIdx.x == 0) finish_instance(P, inst);
}

// packed copy of every instance's breaking keys (then their past keys), arising
// keys and active flags: out = [breaking (nb) | breaking_prev (nb) | arising]
__global__ void k_gather_changes(Pools P, const long long* off, int n, long long nb, unsigned long long* out,
                                 unsigned char* act) {
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const InstDesc& D = P.desc[j];
        const long long b0 = off[3 * j], b1 = off[3 * j + 3];
        const long long a0 = off[3 * j + 1], a1 = off[3 * j + 4];
        const long long k0 = off[3 * j + 2], k1 = off[3 * j + 5];
        for (long long t = threadIdx.x; t < b1 - b0; t += blockDim.x) {
            out[b0 + t] = P.brk[D.edge_off + t];
            out[nb + b0 + t] = P.brk_prev[D.edge_off + t];
        }
        for (long long t = threadIdx.x; t < a1 - a0; t += blockDim.x) out[2 * nb + a0 + t] = P.ari[D.edge_off + t];
        for (long long t = threadIdx.x; t < k1 - k0; t += blockDim.x) act[k0 + t] = P.active[D.comp_off + t];
    }
}

// the same for a list of instances: entry j is instance insts[j], its lists
// span [off[3j + c], off[3j + 3 + c]) of each packed list
__global__ void k_gather_changes_list(Pools P, const int* insts, const long long* off, int n, long long nb,
                                      unsigned long long* out, unsigned char* act) {
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const InstDesc& D = P.desc[insts[j]];
        const long long b0 = off[3 * j], b1 = off[3 * j + 3];
        const long long a0 = off[3 * j + 1], a1 = off[3 * j + 4];
        const long long k0 = off[3 * j + 2], k1 = off[3 * j + 5];
        for (long long t = threadIdx.x; t < b1 - b0; t += blockDim.x) {
            out[b0 + t] = P.brk[D.edge_off + t];
            out[nb + b0 + t] = P.brk_prev[D.edge_off + t];
        }
        for (long long t = threadIdx.x; t < a1 - a0; t += blockDim.x) out[2 * nb + a0 + t] = P.ari[D.edge_off + t];
        for (long long t = threadIdx.x; t < k1 - k0; t += blockDim.x) act[k0 + t] = P.active[D.comp_off + t];
    }
}

void launch_gather_changes_list(cudaStream_t s, const Pools& P, const int* insts, const long long* off, int n,
                                long long nb, unsigned long long* out, unsigned char* act) {
    k_gather_changes_list<<<n < 1024 ? n : 1024, 256, 0, s>>>(P, insts, off, n, nb, out, act);
}

void launch_gather_changes(cudaStream_t s, const Pools& P, const long long* off, int n, long long nb,
                           unsigned long long* out, unsigned char* act) {
    k_gather_changes<<<n < 1024 ? n : 1024, 256, 0, s>>>(P, off, n, nb, out, act);
}

void launch_graph_prep(const Launch& L) {
    launch_plan(L, 0, ends_bit(SCAN_DEG));
}

void launch_graph_csr(const Launch& L) {
    launch_scan(L, SCAN_DEG);
    launch_step(L, k_csr_scatter, dim3(L.grid_wide), dim3(256), L.P, L.T);
    launch_step(L, k_csr_sort, dim3(L.grid_wide), dim3(256), L.P, L.T);
}

void launch_graph_match(const Launch& L) {
    const int g = L.grid_wide;
    if (L.centroid_match) launch_step(L, k_match_kin, dim3(g), dim3(256), L.P, L.T);
    launch_step(L, k_match_best, dim3(g), dim3(256), L.P, L.T);
    launch_step(L, k_match_phi, dim3(g), dim3(256), L.P, L.T);
}

// The translation reads the past frame's CSR, which in a frame sequence is the
// now-frame CSR of the previous instance built in this step: the row
// comparison follows both the match and the CSR chain.
void launch_graph_flips(const Launch& L) {
    const int g = L.grid_wide;
    launch_step(L, k_flip_count, dim3(g), dim3(256), L.P, L.T);
    launch_plan(L, 0, ends_bit(SCAN_FLIPS) | ends_bit(SCAN_FLIPS_A), pre_bit(PRE_FB) | pre_bit(PRE_FA));
    launch_scan2(L, SCAN_FLIPS, SCAN_FLIPS_A);
    launch_step(L, k_flip_write, dim3(g), dim3(256), L.P, L.T);
    if (L.events) launch_step(L, k_events, dim3(g), dim3(256), L.P, L.T);
}

// the CSR and match chains when they run on two forked streams (the prefix
// arrays each writes are disjoint; K and K_past prefixes are final since the
// bubble stage)
void launch_graph_csr_chain(const Launch& L) {
    launch_plan(L, 0, ends_bit(SCAN_DEG), pre_bit(PRE_E));
    launch_graph_csr(L);
}
void launch_graph_match_chain(const Launch& L) {
    launch_plan(L, 0, ENDS_NONE, pre_bit(PRE_O));
    launch_graph_match(L);
}

void launch_graph_inst(const Launch& L) {
    launch_step(L, k_graph_inst_a, dim3(L.T.n_act), dim3(GI_THREADS), L.P, L.T);
    launch_step(L, k_graph_inst_b, dim3(L.T.n_act), dim3(GI_THREADS), L.P, L.T);
}

void launch_begin(const Launch& L) {
    launch_step(L, k_step_begin, dim3(1), dim3(256), L.P, L.T);
}
void launch_finish(const Launch& L) {
    launch_step(L, k_step_finish, dim3(1), dim3(256), L.P, L.T);
}

}  // namespace vd
