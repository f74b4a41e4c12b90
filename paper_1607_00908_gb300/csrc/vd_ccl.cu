// Bubble identification (Section 3.1 of the paper): threshold, periodic
// 4-connected labelling with canonical ids, sizes and centres of mass in
// 1/1024-site fixed point, the centroid bucket grid, and the per-site label
// pass that also builds the past/now overlap histogram (Section 3.2.3).
//
// Labelling works on 64 x 32 tiles. Pass A reads the field once (vector
// loads), stores the foreground bits (1 bit per site), runs a union-find in
// shared memory and emits one "piece" per tile-local component with its size
// and coordinate sums relative to its first site, plus the piece ids along the
// four tile borders. Pieces are then merged across tile borders (periodic) by
// a global union-find whose root is the piece with the smallest first site, so
// the root of every bubble is the bubble's smallest linear index; bubble ids
// are the ranks of those roots (a scan over a root bitmap). The label pass
// re-runs the tile union-find from the stored bits (instead of re-reading the
// field) and writes final labels.
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

__device__ __forceinline__ unsigned long long row_bits(const unsigned (*s_bits)[2], int r) {
    return (unsigned long long)s_bits[r][0] | ((unsigned long long)s_bits[r][1] << 32);
}

// Called by all TTHREADS threads. Thread t owns row t/8, sites 8*(t%8) .. +7.
// On return s_par[i] is the smallest tile-local index of site i's component
// (i itself for a root) for foreground sites, -1 for background sites.
__device__ void tile_union_find(const unsigned (*s_bits)[2], int* s_par) {
    const int r = threadIdx.x >> 3, sg = threadIdx.x & 7;
    const unsigned long long row = row_bits(s_bits, r);
    const unsigned seg = (unsigned)(row >> (sg * 8)) & 0xFFu;
    const int base = r * TW + sg * 8;
    int rs = -1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((seg >> i) & 1u) {
            if (rs < 0) rs = base + i;
            s_par[base + i] = rs;
        } else {
            rs = -1;
            s_par[base + i] = -1;
        }
    }
    __syncthreads();
    if (sg > 0 && (seg & 1u) && ((row >> (sg * 8 - 1)) & 1ull)) uf_union(s_par, base, base - 1);
    if (r > 0) {
        const unsigned long long up = row_bits(s_bits, r - 1);
        const unsigned vm = seg & ((unsigned)(up >> (sg * 8)) & 0xFFu);
        unsigned starts = vm & ~(vm << 1);
        while (starts) {
            const int i = __ffs(starts) - 1;
            starts &= starts - 1;
            uf_union(s_par, base + i, base + i - TW);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if ((seg >> i) & 1u) s_par[base + i] = uf_find(s_par, base + i);
    __syncthreads();
}

// block exclusive scan of one int per thread (TTHREADS threads); returns the
// thread's exclusive prefix and writes the block total to *total
__device__ __forceinline__ int block_excl_scan(int x, int* s_tmp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    int pre = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        int t = s_tmp[w];
        if (w < warp) pre += t;
        tot += t;
    }
    *total = tot;
    __syncthreads();
    return pre + inc - x;
}

// load the tile's foreground bits from the global bitmask
__device__ __forceinline__ void load_tile_bits(const Pools& P, const InstDesc& D, int x0, int y0,
                                               unsigned (*s_bits)[2]) {
    for (int k = threadIdx.x; k < TH * 2; k += blockDim.x) {
        const int r = k >> 1, h = k & 1;
        const int y = y0 + r;
        const int wx = (x0 >> 5) + h;
        unsigned w = 0;
        if (y < D.Ly && wx < D.wpr) w = P.fgbits[D.word_off + (long long)y * D.wpr + wx];
        s_bits[r][h] = w;
    }
    __syncthreads();
}

__device__ __forceinline__ bool is_fg(float v, float thr, int pol) {
    return pol > 0 ? (v > thr) : (v < thr);
}

// ---------------------------------------------------------------------------
// Pass A: threshold + tile union-find + pieces + borders
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(TTHREADS) void k_ccl_tiles(Pools P, StepTable T) {
    __shared__ unsigned s_bits[TH][2];
    __shared__ int s_par[TSITES];
    __shared__ int s_nsv[TSITES];   // (n << 16) | sum of (y - y_root), later piece id
    __shared__ int s_su[TSITES];    // sum of (x - x_root)
    __shared__ int s_tmp[TTHREADS / 32];
    __shared__ int s_base;

    const int b = blockIdx.x;
    const int a = seg_of_int(T.tileA_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileA_pre[a];
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const int r = threadIdx.x >> 3, sg = threadIdx.x & 7;
    const int y = y0 + r, xs = x0 + sg * 8;

    // 1. threshold 8 sites per thread
    unsigned bits8 = 0;
    if (y < D.Ly && xs < D.Lx) {
        const float* f = S.field + (long long)y * S.pitch + xs;
        if (xs + 8 <= D.Lx && ((reinterpret_cast<uintptr_t>(f) & 15u) == 0)) {
            const float4 u = __ldcs(reinterpret_cast<const float4*>(f));
            const float4 w = __ldcs(reinterpret_cast<const float4*>(f) + 1);
            bits8 = (unsigned)is_fg(u.x, D.thr, D.pol) | ((unsigned)is_fg(u.y, D.thr, D.pol) << 1) |
                    ((unsigned)is_fg(u.z, D.thr, D.pol) << 2) | ((unsigned)is_fg(u.w, D.thr, D.pol) << 3) |
                    ((unsigned)is_fg(w.x, D.thr, D.pol) << 4) | ((unsigned)is_fg(w.y, D.thr, D.pol) << 5) |
                    ((unsigned)is_fg(w.z, D.thr, D.pol) << 6) | ((unsigned)is_fg(w.w, D.thr, D.pol) << 7);
        } else {
            for (int i = 0; i < 8; ++i)
                if (xs + i < D.Lx && is_fg(__ldcs(f + i), D.thr, D.pol)) bits8 |= 1u << i;
        }
    }
    // gather the row's two 32-bit words (lanes 8r..8r+3 and 8r+4..8r+7)
    unsigned wv = bits8 << (8 * (sg & 3));
    wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
    wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
    if ((sg & 3) == 0) {
        s_bits[r][sg >> 2] = wv;
        const int wx = (x0 >> 5) + (sg >> 2);
        if (y < D.Ly && wx < D.wpr) P.fgbits[D.word_off + (long long)y * D.wpr + wx] = wv;
    }
    for (int k = threadIdx.x; k < TSITES; k += TTHREADS) {
        s_nsv[k] = 0;
        s_su[k] = 0;
    }
    __syncthreads();

    // 2. tile union-find
    tile_union_find(s_bits, s_par);

    // 3. piece sums, aggregated over runs of equal root within the thread
    const int base = r * TW + sg * 8;
    {
        int cur = -1, cnt = 0, su = 0;
        int nroots = 0;
        for (int i = 0; i < 8; ++i) {
            const int p = s_par[base + i];
            if (p == base + i) ++nroots;
            if (p != cur) {
                if (cur >= 0) {
                    const int dv = r - (cur / TW);
                    atomicAdd(&s_nsv[cur], (cnt << 16) + cnt * dv);
                    atomicAdd(&s_su[cur], su);
                }
                cur = p;
                cnt = 0;
                su = 0;
            }
            if (p >= 0) {
                ++cnt;
                su += (sg * 8 + i) - (p % TW);
            }
        }
        if (cur >= 0) {
            const int dv = r - (cur / TW);
            atomicAdd(&s_nsv[cur], (cnt << 16) + cnt * dv);
            atomicAdd(&s_su[cur], su);
        }
        __syncthreads();

        // 4. roots in raster order -> piece ids
        int m;
        const int rank0 = block_excl_scan(nroots, s_tmp, &m);
        if (threadIdx.x == 0) {
            int bse = atomicAdd(&P.g->n_pieces, m);
            if (bse + m > P.piece_cap) {
                atomicOr(&P.g->err, ERR_PIECE_CAP);
                atomicOr(&P.st[inst].err, ERR_PIECE_CAP);
                bse = -1;
            }
            s_base = bse;
            P.tile_pbase[D.tile_off + t] = bse;
            P.tile_pcnt[D.tile_off + t] = m;
        }
        __syncthreads();
        const int pbase = s_base;
        int rk = rank0;
        for (int i = 0; i < 8; ++i) {
            const int li = base + i;
            if (s_par[li] == li) {
                const int nsv = s_nsv[li];
                int pid = -1;
                if (pbase >= 0) {
                    pid = pbase + rk;
                    P.p_q[pid] = (y0 + r) * D.Lx + x0 + sg * 8 + i;
                    P.p_inst[pid] = inst;
                    P.p_n[pid] = nsv >> 16;
                    P.p_sv[pid] = nsv & 0xFFFF;
                    P.p_su[pid] = s_su[li];
                    P.p_parent[pid] = pid;
                    P.p_accn[pid] = 0;
                    P.p_accx[pid] = 0;
                    P.p_accy[pid] = 0;
                }
                ++rk;
                s_nsv[li] = pid;   // only this thread touches a root's slot
            }
        }
    }
    __syncthreads();

    // 5. borders: [0,TH) left col, [TH,2TH) right col, [2TH,2TH+TW) top row, [.., +TW) bottom row
    const int ncols = min(TW, D.Lx - x0), nrows = min(TH, D.Ly - y0);
    int* bd = P.border + D.border_off + (long long)t * BORDER;
    for (int k = threadIdx.x; k < BORDER; k += TTHREADS) {
        int lx, ly;
        if (k < TH) { ly = k; lx = 0; }
        else if (k < 2 * TH) { ly = k - TH; lx = ncols - 1; }
        else if (k < 2 * TH + TW) { lx = k - 2 * TH; ly = 0; }
        else { lx = k - 2 * TH - TW; ly = nrows - 1; }
        int v = -1;
        if (lx < ncols && ly < nrows) {
            const int p = s_par[ly * TW + lx];
            if (p >= 0) v = s_nsv[p];
        }
        bd[k] = v;
    }
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

__device__ __forceinline__ void punion(const Pools& P, int a, int b) {
    for (;;) {
        a = pfind(P.p_parent, a);
        b = pfind(P.p_parent, b);
        if (a == b) return;
        const int qa = P.p_q[a], qb = P.p_q[b];
        if (qa > qb) { const int t = a; a = b; b = t; }
        if (atomicCAS(&P.p_parent[b], b, a) == b) return;
    }
}

__global__ void k_ccl_merge(Pools P, StepTable T, int total) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int a = seg_of_int(T.merge_pre, T.n_act, g);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const int loc = g - T.merge_pre[a];
    const int t = loc / (TW + TH), j = loc % (TW + TH);
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int* bd = P.border + D.border_off;
    int pa, pb;
    if (j < TH) {
        const int tn = ty * D.ntx + (tx + 1) % D.ntx;
        pa = bd[(long long)t * BORDER + TH + j];
        pb = bd[(long long)tn * BORDER + j];
    } else {
        const int k = j - TH;
        const int tn = ((ty + 1) % D.nty) * D.ntx + tx;
        pa = bd[(long long)t * BORDER + 2 * TH + TW + k];
        pb = bd[(long long)tn * BORDER + 2 * TH + k];
    }
    if (pa >= 0 && pb >= 0) punion(P, pa, pb);
}

// root of each piece; roots are counted per instance and marked in the root bitmap
__global__ void k_ccl_flatten(Pools P) {
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        const int r = pfind(P.p_parent, pid);
        P.p_parent[pid] = r;
        if (r == pid) {
            const int inst = P.p_inst[pid];
            const InstDesc& D = P.desc[inst];
            const int q = P.p_q[pid];
            const int y = q / D.Lx, x = q - y * D.Lx;
            atomicOr(&P.rootbits[D.word_off + (long long)y * D.wpr + (x >> 5)], 1u << (x & 31));
            atomicAdd(&P.st[inst].K, 1);
        }
    }
}

// bubble ids of roots; exact coordinate sums relative to the bubble's first site
__global__ void k_comp_accum(Pools P) {
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const int r = P.p_parent[pid];
        const int q = P.p_q[pid];
        const int yq = q / D.Lx, xq = q - yq * D.Lx;
        if (r == pid) {
            const long long w = D.word_off + (long long)yq * D.wpr + (xq >> 5);
            const int c = P.rankpre[w] + __popc(P.rootbits[w] & ((1u << (xq & 31)) - 1u));
            P.p_comp[pid] = c;
            if (c < D.comp_cap) P.comp_root[D.comp_off + c] = pid;
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
            const int w = atomicAdd(&P.g->n_wide, 1);
            P.wide[w] = pid;
        }
    }
}

// exact per-site sums for pieces whose minimum image is not a single shift
__global__ __launch_bounds__(TTHREADS) void k_comp_wide(Pools P) {
    __shared__ unsigned s_bits[TH][2];
    __shared__ int s_par[TSITES];
    __shared__ long long s_red[3][TTHREADS / 32];
    const int nw = P.g->n_wide;
    for (int w = blockIdx.x; w < nw; w += gridDim.x) {
        const int pid = P.wide[w];
        const int inst = P.p_inst[pid];
        const InstDesc D = P.desc[inst];
        const int q = P.p_q[pid];
        const int yq = q / D.Lx, xq = q - yq * D.Lx;
        const int x0 = (xq / TW) * TW, y0 = (yq / TH) * TH;
        const int r = P.p_parent[pid];
        const int qr = P.p_q[r];
        const int yr = qr / D.Lx, xr = qr - yr * D.Lx;
        load_tile_bits(P, D, x0, y0, s_bits);
        tile_union_find(s_bits, s_par);
        const int lq = (yq - y0) * TW + (xq - x0);
        long long n = 0, sx = 0, sy = 0;
        const int rr = threadIdx.x >> 3, sg = threadIdx.x & 7;
        for (int i = 0; i < 8; ++i) {
            const int li = rr * TW + sg * 8 + i;
            if (s_par[li] == lq) {
                ++n;
                sx += wrap_ll((x0 + sg * 8 + i) - xr, D.Lx);
                sy += wrap_ll((y0 + rr) - yr, D.Ly);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            n += __shfl_xor_sync(0xffffffffu, n, o);
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { s_red[0][warp] = n; s_red[1][warp] = sx; s_red[2][warp] = sy; }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long a0 = 0, a1 = 0, a2 = 0;
            for (int k = 0; k < TTHREADS / 32; ++k) { a0 += s_red[0][k]; a1 += s_red[1][k]; a2 += s_red[2][k]; }
            atomicAdd((unsigned long long*)&P.p_accn[r], (unsigned long long)a0);
            atomicAdd((unsigned long long*)&P.p_accx[r], (unsigned long long)a1);
            atomicAdd((unsigned long long*)&P.p_accy[r], (unsigned long long)a2);
        }
        __syncthreads();
    }
}

// Q10 centroids of bubbles; bucket counts; clear the root bitmap for the next step
__global__ void k_comp_final(Pools P) {
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        if (P.p_parent[pid] != pid) continue;
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const InstState& S = P.st[inst];
        const int q = P.p_q[pid];
        const int yq = q / D.Lx, xq = q - yq * D.Lx;
        P.rootbits[D.word_off + (long long)yq * D.wpr + (xq >> 5)] = 0u;
        const int c = P.p_comp[pid];
        if (c >= D.comp_cap) continue;
        const long long nn = P.p_accn[pid];
        const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
        // round half up: floor((2p + n) / 2n) with p = 1024 * S
        long long cx = (long long)Q * xq + floordiv_ll(2 * (long long)Q * P.p_accx[pid] + nn, 2 * nn);
        long long cy = (long long)Q * yq + floordiv_ll(2 * (long long)Q * P.p_accy[pid] + nn, 2 * nn);
        cx %= MX; if (cx < 0) cx += MX;
        cy %= MY; if (cy < 0) cy += MY;
        P.cq[D.comp_off + c] = make_int2((int)cx, (int)cy);
        const int bx = (int)(cx / Q) / S.B, by = (int)(cy / Q) / S.B;
        atomicAdd(&P.bcnt[D.bucket_off + (long long)by * S.nbx + bx], 1);
    }
}

// counting-sort scatter of centroids into bucket order (counts return to zero)
__global__ void k_bucket_scatter(Pools P) {
    const int n = min(P.g->n_pieces, P.piece_cap);
    for (int pid = blockIdx.x * blockDim.x + threadIdx.x; pid < n; pid += gridDim.x * blockDim.x) {
        if (P.p_parent[pid] != pid) continue;
        const int inst = P.p_inst[pid];
        const InstDesc& D = P.desc[inst];
        const InstState& S = P.st[inst];
        const int c = P.p_comp[pid];
        if (c >= D.comp_cap) continue;
        const int2 v = P.cq[D.comp_off + c];
        const long long bk = D.bucket_off + (long long)((v.y / Q) / S.B) * S.nbx + (v.x / Q) / S.B;
        const int pos = P.boff[bk] + atomicSub(&P.bcnt[bk], 1) - 1;
        P.bcq[D.comp_off + pos] = v;
        P.bid[D.comp_off + pos] = c;
    }
}

// ---------------------------------------------------------------------------
// Label pass: final labels from the stored bits; overlap histogram with the
// previous frame's labels (Section 3.2.3)
// ---------------------------------------------------------------------------
constexpr int OSET = 256;

__device__ __forceinline__ void ovl_global_insert(const Pools& P, const InstDesc& D, int inst,
                                                  unsigned long long key, unsigned cnt) {
    unsigned long long* H = P.ohash + D.ohash_off;
    unsigned* V = P.oval + D.ohash_off;
    unsigned h = (unsigned)hash64(key) & (unsigned)D.ohash_mask;
    for (int probe = 0; probe <= D.ohash_mask; ++probe) {
        const unsigned long long k = atomicCAS(&H[h], EMPTY_KEY, key);
        if (k == EMPTY_KEY || k == key) {
            atomicAdd(&V[h], cnt);
            if (k == EMPTY_KEY) {
                const int idx = atomicAdd(&P.st[inst].n_ovl, 1);
                if (idx < D.ovl_cap) P.olist[D.ovl_off + idx] = (int)h;
                else atomicOr(&P.st[inst].err, ERR_OVL_CAP);
            }
            return;
        }
        h = (h + 1) & (unsigned)D.ohash_mask;
    }
    atomicOr(&P.st[inst].err, ERR_OVL_CAP);
}

__device__ __forceinline__ void ovl_add(unsigned long long* s_key, unsigned* s_cnt, const Pools& P,
                                        const InstDesc& D, int inst, unsigned long long key, unsigned cnt) {
    unsigned h = (unsigned)hash64(key) & (OSET - 1);
    for (int probe = 0; probe < OSET; ++probe) {
        const unsigned long long k = atomicCAS(&s_key[h], EMPTY_KEY, key);
        if (k == EMPTY_KEY || k == key) {
            atomicAdd(&s_cnt[h], cnt);
            return;
        }
        h = (h + 1) & (OSET - 1);
    }
    ovl_global_insert(P, D, inst, key, cnt);   // shared set full
}

__global__ __launch_bounds__(TTHREADS) void k_labels(Pools P, StepTable T) {
    __shared__ unsigned s_bits[TH][2];
    __shared__ int s_par[TSITES];
    __shared__ int s_comp[TSITES];
    __shared__ int s_tmp[TTHREADS / 32];
    __shared__ unsigned long long s_key[OSET];
    __shared__ unsigned s_cnt[OSET];

    const int b = blockIdx.x;
    const int a = seg_of_int(T.tileA_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileA_pre[a];
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int x0 = tx * TW, y0 = ty * TH;
    const int now = S.slot ^ 1;
    const bool with_prev = S.has_prev != 0;

    for (int k = threadIdx.x; k < OSET; k += TTHREADS) {
        s_key[k] = EMPTY_KEY;
        s_cnt[k] = 0;
    }
    load_tile_bits(P, D, x0, y0, s_bits);
    tile_union_find(s_bits, s_par);

    const int r = threadIdx.x >> 3, sg = threadIdx.x & 7;
    const int base = r * TW + sg * 8;
    int nroots = 0;
    for (int i = 0; i < 8; ++i) nroots += (s_par[base + i] == base + i);
    int m;
    int rk = block_excl_scan(nroots, s_tmp, &m);
    const int pbase = P.tile_pbase[D.tile_off + t];
    for (int i = 0; i < 8; ++i) {
        const int li = base + i;
        if (s_par[li] == li) {
            int c = -1;
            if (pbase >= 0) c = P.p_comp[P.p_parent[pbase + rk]];
            s_comp[li] = c;
            ++rk;
        }
    }
    __syncthreads();

    const int y = y0 + r, xs = x0 + sg * 8;
    if (y < D.Ly && xs < D.Lx) {
        int lab[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int p = s_par[base + i];
            lab[i] = p >= 0 ? s_comp[p] : -1;
        }
        int* out = P.labels[now] + D.site_off + (long long)y * D.Lx + xs;
        const int* prv = P.labels[now ^ 1] + D.site_off + (long long)y * D.Lx + xs;
        int pl[8];
        const bool vec = (xs + 8 <= D.Lx) && ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
        if (vec) {
            reinterpret_cast<int4*>(out)[0] = make_int4(lab[0], lab[1], lab[2], lab[3]);
            reinterpret_cast<int4*>(out)[1] = make_int4(lab[4], lab[5], lab[6], lab[7]);
            if (with_prev) {
                const int4 u = __ldcs(reinterpret_cast<const int4*>(prv));
                const int4 w = __ldcs(reinterpret_cast<const int4*>(prv) + 1);
                pl[0] = u.x; pl[1] = u.y; pl[2] = u.z; pl[3] = u.w;
                pl[4] = w.x; pl[5] = w.y; pl[6] = w.z; pl[7] = w.w;
            }
        } else {
            for (int i = 0; i < 8; ++i) {
                if (xs + i < D.Lx) {
                    out[i] = lab[i];
                    pl[i] = with_prev ? prv[i] : -1;
                } else {
                    pl[i] = -1;
                }
            }
        }
        if (with_prev) {
            unsigned long long cur = EMPTY_KEY;
            unsigned cnt = 0;
            for (int i = 0; i < 8; ++i) {
                const bool inb = (xs + i < D.Lx);
                const bool both = inb && lab[i] >= 0 && pl[i] >= 0;
                const unsigned long long key =
                    both ? (((unsigned long long)(unsigned)pl[i] << 32) | (unsigned)lab[i]) : EMPTY_KEY;
                if (key != cur) {
                    if (cur != EMPTY_KEY) ovl_add(s_key, s_cnt, P, D, inst, cur, cnt);
                    cur = key;
                    cnt = 0;
                }
                if (both) ++cnt;
            }
            if (cur != EMPTY_KEY) ovl_add(s_key, s_cnt, P, D, inst, cur, cnt);
        }
    }
    if (with_prev) {
        __syncthreads();
        for (int k = threadIdx.x; k < OSET; k += TTHREADS)
            if (s_key[k] != EMPTY_KEY) ovl_global_insert(P, D, inst, s_key[k], s_cnt[k]);
    }
}

void launch_ccl_tiles(const Launch& L) {
    k_ccl_tiles<<<L.total_tilesA, TTHREADS, 0, L.s>>>(L.P, L.T);
    ++*L.nlaunch;
}

void launch_ccl_rest(const Launch& L) {
    if (L.total_merge > 0) {
        k_ccl_merge<<<(L.total_merge + 255) / 256, 256, 0, L.s>>>(L.P, L.T, L.total_merge);
        ++*L.nlaunch;
    }
    k_ccl_flatten<<<L.grid_items, 256, 0, L.s>>>(L.P);
    ++*L.nlaunch;
    launch_plan(L, 1);
    launch_scan(L, SCAN_ROOTBITS);
    k_comp_accum<<<L.grid_items, 256, 0, L.s>>>(L.P);
    ++*L.nlaunch;
    k_comp_wide<<<L.grid_items, TTHREADS, 0, L.s>>>(L.P);
    ++*L.nlaunch;
    k_comp_final<<<L.grid_items, 256, 0, L.s>>>(L.P);
    ++*L.nlaunch;
    launch_scan(L, SCAN_BUCKETS);
    k_bucket_scatter<<<L.grid_items, 256, 0, L.s>>>(L.P);
    ++*L.nlaunch;
}

void launch_labels(const Launch& L) {
    k_labels<<<L.total_tilesA, TTHREADS, 0, L.s>>>(L.P, L.T);
    ++*L.nlaunch;
}

}  // namespace vd
