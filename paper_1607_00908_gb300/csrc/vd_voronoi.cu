// Digital Voronoi colouring (Section 3.2.1) and Delaunay links (Section 3.2.2).
//
// owner(s) = argmin_i |1024*s - c_i|^2 over all bubble centres (exact int64,
// minimum image on the torus, ties to the smallest label). The paper computes
// this by scanning every centre from every site; here each 64 x 32 tile first
// collects a provably complete candidate set from a bucket grid of centres,
// and each patch of it (8 x 8 sites by default; the layout is a launch shape)
// keeps only the centres that can own one of its sites:
//   U_p   = min over scanned centres of an upper bound of their largest
//           distance to patch p (so every site of p has a centre within U_p),
//   keep  = centres whose smallest distance to the patch is <= U_p,
// scanning rings of buckets around the tile until the unscanned region is
// farther than sqrt(max_p U_p). Each site then scans only its patch's kept
// candidates.
//
// Links: a link {a, b} joins owners that meet where a site and its +x or +y
// neighbour differ, and for a 2x2 plaquette with four distinct owners the
// diagonal chosen by the exact incircle test (int128). Each tile emits every
// owner pair that meets in it at least once (one key per boundary piece, not
// per site); the keys are then inserted into a global hash that also counts
// each label's degree.
#include "vd_internal.cuh"

namespace vd {

// distance from a point (offset d of the point from the interval start, already
// reduced to [-M/2, M/2)) to an interval [0, W] on a ring of length M
__device__ __forceinline__ long long ring_mindist(long long d, long long W, long long M) {
    long long best = LLONG_MAX;
#pragma unroll
    for (int k = -1; k <= 1; ++k) {
        const long long t = d + k * M;
        const long long v = t < 0 ? -t : (t > W ? t - W : 0);
        best = v < best ? v : best;
    }
    return best;
}

__device__ __forceinline__ long long wrapM(long long d, long long M) {
    // d in (-M, M] -> [-M/2, M/2)
    const long long h = M >> 1;
    if (d >= h) d -= M;
    else if (d < -h) d += M;
    return d;
}

__device__ __forceinline__ int sgn128(__int128 v) { return (v > 0) - (v < 0); }

// diagonal of a four-colour plaquette A B / D C (cyclic A, B, C, D)
__device__ unsigned long long plaquette_key(int A, int B, int C, int D, const int2* cq, long long MX,
                                            long long MY) {
    const int2 a = cq[A], b = cq[B], c = cq[C], d = cq[D];
    const long long bx = wrapM((long long)b.x - a.x, MX), by = wrapM((long long)b.y - a.y, MY);
    const long long cx = wrapM((long long)c.x - a.x, MX), cy = wrapM((long long)c.y - a.y, MY);
    const long long dx = wrapM((long long)d.x - a.x, MX), dy = wrapM((long long)d.y - a.y, MY);
    // a at the origin
    const __int128 orient = (__int128)bx * cy - (__int128)by * cx;
    const __int128 adx = -dx, ady = -dy;
    const __int128 bdx = bx - dx, bdy = by - dy;
    const __int128 cdx = cx - dx, cdy = cy - dy;
    const __int128 inc = (adx * adx + ady * ady) * (bdx * cdy - cdx * bdy) +
                         (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy) +
                         (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady);
    const int s = sgn128(inc) * sgn128(orient);
    const int mBD = B < D ? B : D, mAC = A < C ? A : C;
    if (s > 0 || (s == 0 && mBD < mAC)) return edge_key(B, D);
    return edge_key(A, C);
}

__device__ __forceinline__ void edge_global_insert(const Pools& P, const InstDesc& D, int inst,
                                                   unsigned long long key) {
    unsigned long long* H = P.ehash + D.ehash_off;
    const unsigned mask = dyn_mask(D.ehash_mask, 16ll * P.st[inst].K + 64);
    unsigned h = (unsigned)hash64(key) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = atomicCAS(&H[h], EMPTY_KEY, key);
        if (k == EMPTY_KEY) {
            const int idx = warp_fetch_inc(&P.st[inst].n_edge_list);
            if (idx < D.edge_cap) {
                P.elist[D.edge_off + idx] = (int)h;
            } else if (!(atomicOr(&P.st[inst].err, ERR_EDGE_CAP) & (ERR_EDGE_CAP | ERR_OVL_CAP))) {
                atomicAdd(&P.g->lists_over, 1);
            }
            atomicAdd(&P.deg[D.comp_off + (int)(key >> 32)], 1);
            atomicAdd(&P.deg[D.comp_off + (int)(key & 0xffffffffu)], 1);
            return;
        }
        if (k == key) return;
        h = (h + 1) & mask;
    }
    if (!(atomicOr(&P.st[inst].err, ERR_EDGE_CAP) & (ERR_EDGE_CAP | ERR_OVL_CAP))) atomicAdd(&P.g->lists_over, 1);
}


constexpr int VWARPS = 2;        // tiles per block, one warp each
constexpr int WSCAN = 384;       // per-warp list of scanned centres
constexpr int KMAX = 16;         // kept centres listed per patch (more: exact over every scanned centre)

// Patch layouts of the owner kernel: a 64 x 32 tile is cut into NP patches of
// PW x PH sites. Lane p computes the bound and the kept list of patch p
// (NP <= 32); in the site phase every lane takes SPL sites of one column of a
// patch (column lane % PW, rows from (lane / PW) * SPL).
template <int PW_, int PH_>
struct VLayout {
    static constexpr int PW = PW_, PH = PH_;
    static constexpr int NPX = TW / PW, NPY = TH / PH, NP = NPX * NPY;
    static constexpr int SPL = PW * PH / 32;
    // lanes per patch in the bound and kept-list passes: lane l serves patch
    // l % NP and takes every LPP-th scanned centre
    static constexpr int LPP = 32 / NP;
    // resident blocks per SM the registers are sized for (measured: 8x8
    // patches run fastest at 72 registers, the others at 64)
    static constexpr int MINB = (PW == 8 && PH == 8) ? 14 : 16;
    static_assert(TW % PW == 0 && TH % PH == 0 && NP <= 32 && 32 % NP == 0 && 32 % PW == 0 && SPL >= 1 &&
                      (32 / PW) * SPL == PH,
                  "patch layout");
};

// The integer held in a list coordinate (an integer in [-2^22, 2^22), exact
// in float32): adding 1.5 * 2^23 places it in [2^23, 2^24), where the float's
// low mantissa bits are the integer plus 2^22 -- two full-rate instructions
// instead of a conversion.
__device__ __forceinline__ int list_int(float v) { return __float_as_int(v + 12582912.f) - 0x4B400000; }
// and the converse, for integers in [-2^22, 2^22)
__device__ __forceinline__ float int_to_f(int i) { return __int_as_float(0x4B400000 + i) - 12582912.f; }

// Exact owner over a kept list with int64 distances (coordinates relative to
// the tile origin, no wrap needed), ties to the smallest label. kk maps list
// positions to entries.
__device__ __forceinline__ int owner_exact(long long sx, long long sy, const float2* cf, const int* id, const int* kk,
                                           int n) {
    long long best = LLONG_MAX;
    int bi = -1;
    for (int j = 0; j < n; ++j) {
        const int e = kk[j];
        const long long dx = sx - list_int(cf[e].x), dy = sy - list_int(cf[e].y);
        const long long d2 = dx * dx + dy * dy;
        if (d2 < best || (d2 == best && id[e] < bi)) { best = d2; bi = id[e]; }
    }
    return bi;
}

// A scanned centre's coordinate as held in the list: the tile-relative
// minimum image when it lies in [-2^22, 2^22) (exact in float32), else
// +-2^31, which makes the patch bound take the half-period cap for that axis
// (a larger upper bound, still valid); such a tile takes the general path.
__device__ __forceinline__ bool list_exact(int w) { return w >= -(1 << 22) && w < (1 << 22); }
__device__ __forceinline__ float list_coord(int w) {
    return list_exact(w) ? (float)w : (w > 0 ? 2147483648.f : -2147483648.f);
}

// One warp per 64 x 32 tile (the labelling tiles), no block-level
// synchronisation; two tiles per block.
//  1. Ring search over the bucket grid around the tile: the centres of the
//     rings of buckets are collected in shared memory (one bucket per lane,
//     placed by a prefix sum), starting with the rings within `ring0` sites
//     plus one bucket. Lane p then updates, over the new centres, U_p = the
//     smallest upper bound (float32 rounded up) of a centre's largest squared
//     distance to patch p, so every site of patch p has a centre within
//     sqrt(U_p). The search stops when the unscanned region is farther than
//     sqrt(max_p U_p) from the tile.
//  2. Lane p lists the scanned centres whose smallest squared distance to
//     patch p (rounded down) is <= U_p: the owner of every site of the patch
//     is among them (it is within sqrt(U_p) of the site, hence of the patch,
//     and every such centre was scanned).
//  3. Patch by patch, every lane takes SPL sites: one kept centre owns the
//     whole patch; two are decided by their exact int64 bisector stepped down
//     the column; more are screened in float32 (squared distance with the
//     kept index in the low 6 bits: the two smallest give the nearest and the
//     runner-up) and decided exactly in int64 over the kept list when the two
//     are within 2^-15 relative (truncation 2^-17 + rounding 2^-23 cannot
//     reorder them otherwise), ties to the smallest label.
//  Centres are held in float32 (integers below 2^22, exact), so the bound and
//  list passes run on the FP32 pipe without conversions. A tile whose scanned
//  centres are not minimum images for every site or not exact in float32, or
//  whose scan exceeds WSCAN centres, takes the general path (exact int64 per
//  site over the scanned buckets).
template <int PW, int PH>
__global__ __launch_bounds__(32 * VWARPS, VLayout<PW, PH>::MINB) void k_voronoi(Pools P, StepTable T) {
    using LY = VLayout<PW, PH>;
    constexpr int NPX = LY::NPX, NP = LY::NP, SPL = LY::SPL, LPP = LY::LPP;
    pdl_enter();
    __shared__ float2 s_cf[VWARPS][WSCAN];
    __shared__ int s_id[VWARPS][WSCAN];
    __shared__ __align__(16) int s_kept[VWARPS][NP][KMAX];
    __shared__ int s_nk[VWARPS][NP];
    __shared__ int s_tpre[SEG_CACHE];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int* tpre = seg_table(T.tileA_pre, T.n_act, s_tpre);
    const int b = blockIdx.x * VWARPS + warp;
    if (b >= tpre[T.n_act]) return;
    const int a = seg_of_int(tpre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - tpre[a];
    const int tx = t % D.ntx, ty = t / D.ntx;
    const int Lx = D.Lx, Ly = D.Ly;
    const int x0 = tx * TW, y0 = ty * TH;
    const int ncols = min(TW, Lx - x0), nrows = min(TH, Ly - y0);
    const int K = min(S.K, D.comp_cap);
    int* own = P.owners + D.site_off;
    if (K <= 0) {
        for (int k = lane; k < ncols * nrows; k += 32)
            own[(long long)(y0 + k / ncols) * Lx + x0 + k % ncols] = -1;
        return;
    }

    // ---- 1. ring search over the bucket grid ----
    // Bucket indices are unwrapped (they may run below 0 or past nb-1 by
    // less than one period). Centre positions are stored relative to the
    // tile origin (minimum image, |v| <= M/2 < 2^31).
    const long long MX = (long long)Q * Lx, MY = (long long)Q * Ly;
    const long long X0 = (long long)Q * x0, Y0 = (long long)Q * y0;
    const int hMX = (int)(MX >> 1), hMY = (int)(MY >> 1);
    const int Bk = S.B, nbx = S.nbx, nby = S.nby;
    const int bx0 = x0 / Bk, bx1 = (x0 + ncols - 1) / Bk;
    const int by0 = y0 / Bk, by1 = (y0 + nrows - 1) / Bk;
    const int* boff = P.boff[S.slot ^ 1] + D.bucket_off;
    const int2* bcq = P.bcq[S.slot ^ 1] + D.comp_off;
    const int* bid = P.bid[S.slot ^ 1] + D.comp_off;
    float2* cfs = s_cf[warp];
    int* ids = s_id[warp];
    // this lane's patch; the LPP lanes of a patch split the scanned centres
    const int pp = lane % NP, sub = lane / NP;
    const int ppx = PW * (pp % NPX), ppy = PH * (pp / NPX);
    const bool pvalid = ppx < ncols && ppy < nrows;
    const int pxlo = Q * ppx, pxhi = Q * max(min(ppx + PW, ncols) - 1, ppx);
    const int pylo = Q * ppy, pyhi = Q * max(min(ppy + PH, nrows) - 1, ppy);
    // patch centre and half extent (multiples of Q/2: exact in float32); the
    // largest distance of a point d to the patch along x is |d - mx| + hwx,
    // the smallest max(0, |d - mx| - hwx)
    const float mxf = (float)((pxlo + pxhi) >> 1), hwxf = (float)((pxhi - pxlo) >> 1);
    const float myf = (float)((pylo + pyhi) >> 1), hwyf = (float)((pyhi - pylo) >> 1);
    const float hMXf = __int2float_ru(hMX), hMYf = __int2float_ru(hMY);
    // minimum image for every site of the tile, and exact in float32
    const int WRt = Q * (ncols - 1), HRt = Q * (nrows - 1);
    bool fit = true;
    float Up = INFINITY;
    int qx0 = 0, qx1 = -1, qy0 = 0, qy1 = -1;   // previous round's region
    bool qfx = false, qfy = false, have_prev = false;
    int rx0, rx1, ry0, ry1;
    int n = 0, nb = 0;   // centres scanned so far, and those whose bounds are taken (warp-uniform)
    for (int r = (D.ring0 + Bk - 1) / Bk + 1;; ++r) {
        rx0 = bx0 - r; rx1 = bx1 + r; ry0 = by0 - r; ry1 = by1 + r;
        const bool fx = (rx1 - rx0 + 1) >= nbx, fy = (ry1 - ry0 + 1) >= nby;
        if (fx) { rx0 = 0; rx1 = nbx - 1; }
        if (fy) { ry0 = 0; ry1 = nby - 1; }
        const int wx = rx1 - rx0 + 1, ncell = wx * (ry1 - ry0 + 1);
        for (int kb = 0; kb < ncell; kb += 32) {   // warp-uniform loop
            const int k = kb + lane;
            int jb = 0, je = 0;
            if (k < ncell) {
                const int kr = k / wx;
                const int cu = rx0 + (k - kr * wx), rv = ry0 + kr;
                bool skip = false;
                if (have_prev) {
                    int dxp = cu - qx0, dyp = rv - qy0;
                    if (dxp < 0) dxp += nbx; else if (dxp >= nbx) dxp -= nbx;
                    if (dyp < 0) dyp += nby; else if (dyp >= nby) dyp -= nby;
                    skip = (qfx || dxp <= qx1 - qx0) && (qfy || dyp <= qy1 - qy0);
                }
                if (!skip) {
                    const int cm = cu < 0 ? cu + nbx : (cu >= nbx ? cu - nbx : cu);
                    const int rm = rv < 0 ? rv + nby : (rv >= nby ? rv - nby : rv);
                    const int bk = rm * nbx + cm;
                    jb = boff[bk];
                    je = max(boff[bk + 1], jb);   // offsets of a frame whose scan gave up may decrease
                }
            }
            const int cnt = je - jb;
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int pos = n + inc - cnt;
            n += __shfl_sync(0xffffffffu, inc, 31);
            for (int j = jb; j < je && pos < WSCAN; ++j, ++pos) {
                const int2 cc = bcq[j];
                const int wx = (int)wrapM((long long)cc.x - X0, MX), wy = (int)wrapM((long long)cc.y - Y0, MY);
                fit = fit && wx > WRt - hMX && wy > HRt - hMY && list_exact(wx) && list_exact(wy);
                cfs[pos] = make_float2(list_coord(wx), list_coord(wy));
                ids[pos] = bid[j];
            }
        }
        __syncwarp();
        // this lane's patch bound over the centres of this round
        const int ne = min(n, WSCAN);
        for (int j = nb + sub; j < ne; j += LPP) {
            const float2 c = cfs[j];
            const float tx = fminf(__fadd_ru(fabsf(c.x - mxf), hwxf), hMXf);
            const float ty = fminf(__fadd_ru(fabsf(c.y - myf), hwyf), hMYf);
            Up = fminf(Up, __fadd_ru(__fmul_ru(tx, tx), __fmul_ru(ty, ty)));
        }
#pragma unroll
        for (int o = NP; o < 32; o <<= 1) Up = fminf(Up, __shfl_xor_sync(0xffffffffu, Up, o));
        nb = ne;
        float Umax = pvalid ? Up : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Umax = fmaxf(Umax, __shfl_xor_sync(0xffffffffu, Umax, o));
        if (fx && fy) break;
        // gap between the region and the unscanned buckets (periods handled by
        // one conditional shift: the ranges are narrower than a period here)
        long long g = LLONG_MAX;
        if (!fx) {
            const int lx = rx0 < 0 ? (rx0 + nbx) * Bk - Lx : rx0 * Bk;                    // start of bucket rx0
            const int ex = rx1 >= nbx ? min((rx1 - nbx + 1) * Bk, Lx) + Lx : min((rx1 + 1) * Bk, Lx);   // end of rx1
            g = min((long long)Q * (x0 - lx), (long long)Q * (ex - (x0 + ncols - 1)));
        }
        if (!fy) {
            const int ly = ry0 < 0 ? (ry0 + nby) * Bk - Ly : ry0 * Bk;
            const int ey = ry1 >= nby ? min((ry1 - nby + 1) * Bk, Ly) + Ly : min((ry1 + 1) * Bk, Ly);
            g = min(g, min((long long)Q * (y0 - ly), (long long)Q * (ey - (y0 + nrows - 1))));
        }
        // every unscanned centre is at least g away from every patch; the
        // double product is within 2^-53 of g^2, so the margin makes it exact
        if (g > 0 && (double)g * (double)g > (double)Umax * (1.0 + 1.0 / (1ll << 50))) break;
        qx0 = rx0; qx1 = rx1; qy0 = ry0; qy1 = ry1; qfx = fx; qfy = fy; have_prev = true;
    }

    // The fast path needs every scanned centre's tile-relative position to be
    // its minimum image for every site of the tile (otherwise the distances
    // are not the torus distances) and exact in float32 (in [-2^22, 2^22)).
    const bool over = n > WSCAN;
    const bool bad = __any_sync(0xffffffffu, !fit) || over;

    if (!bad) {
        // ---- 2. kept list of this lane's patch ----
        {
            int* kl = s_kept[warp][pp];
            int nk = 0;   // the same in every lane of the patch
            if constexpr (LPP == 1) {
                for (int j = 0; j < n; ++j) {
                    const float2 c = cfs[j];
                    // exact: integers below 2^23
                    const float exf = fmaxf(fabsf(c.x - mxf) - hwxf, 0.f), eyf = fmaxf(fabsf(c.y - myf) - hwyf, 0.f);
                    if (__fmaf_rd(exf, exf, __fmul_rd(eyf, eyf)) <= Up) {
                        if (nk < KMAX && vd_in(P, CHK_KEPT, j, n)) kl[nk] = j;
                        ++nk;
                    }
                }
            } else {
                // lanes p, p + NP, ... take centres in turn; each keeps its
                // place among the patch's kept centres of the round by ballot
                unsigned same = 0;
#pragma unroll
                for (int k = 0; k < LPP; ++k) same |= 1u << (pp + k * NP);
                const unsigned below = same & ((1u << lane) - 1u);
                for (int j0 = 0; j0 < n; j0 += LPP) {
                    const int j = j0 + sub;
                    bool keep = false;
                    if (j < n) {
                        const float2 c = cfs[j];
                        const float exf = fmaxf(fabsf(c.x - mxf) - hwxf, 0.f),
                                    eyf = fmaxf(fabsf(c.y - myf) - hwyf, 0.f);
                        keep = __fmaf_rd(exf, exf, __fmul_rd(eyf, eyf)) <= Up;
                    }
                    const unsigned kb = __ballot_sync(0xffffffffu, keep);
                    const int at = nk + __popc(kb & below);
                    if (keep && at < KMAX && vd_in(P, CHK_KEPT, j, n)) kl[at] = j;
                    nk += __popc(kb & same);
                }
            }
            if (sub == 0) s_nk[warp][pp] = nk;
        }
        __syncwarp();
        // ---- per-patch set-up of the site phase, once per patch (in the
        // unused part of its kept row) instead of once per lane: the owner of
        // a one-centre patch; for two centres their exact bisector,
        // d(s,c1)^2 - d(s,c2)^2 = 2 s.(c2 - c1) + |c1|^2 - |c2|^2, as its value
        // at the patch origin and its steps per site along x and y (int64,
        // tile-relative minimum images), and the two labels ----
        if (sub == 0) {
            const int nk = s_nk[warp][pp];
            int* kl = s_kept[warp][pp];
            if (nk == 1) {
                kl[2] = ids[kl[0]];
            } else if (nk == 2) {
                const int e1 = kl[0], e2 = kl[1];
                const long long c1x = list_int(cfs[e1].x), c1y = list_int(cfs[e1].y);
                const long long c2x = list_int(cfs[e2].x), c2y = list_int(cfs[e2].y);
                const long long axq = 2 * (c2x - c1x) * Q, ayq = 2 * (c2y - c1y) * Q;
                long long* co = reinterpret_cast<long long*>(kl + 4);
                co[0] = axq * ppx + ayq * ppy + (c1x * c1x + c1y * c1y) - (c2x * c2x + c2y * c2y);
                co[1] = axq;
                co[2] = ayq;
                kl[2] = ids[e1];
                kl[3] = ids[e2];
            }
        }
        __syncwarp();
        // ---- 3. nearest kept centre for every site, patch by patch ----
        int* ownT = own + (long long)y0 * Lx + x0;   // rows of the tile: row offsets below 2^26
        const int c = lane % PW, rb = (lane / PW) * SPL;
#pragma unroll 1
        for (int p = 0; p < NP; ++p) {
            const int pxo = PW * (p % NPX), pyo = PH * (p / NPX);
            if (pxo >= ncols || pyo >= nrows) continue;   // warp-uniform
            const int pw = min(PW, ncols - pxo), ph = min(PH, nrows - pyo);
            const int nk = s_nk[warp][p];
            const int* kk = s_kept[warp][p];
            if (c < pw && rb < ph) {
                const int sx = pxo + c;
                int o[SPL];
                if (nk == 1) {
                    // one candidate owns the whole patch
                    const int o1 = kk[2];
#pragma unroll
                    for (int k = 0; k < SPL; ++k) o[k] = o1;
                } else if (nk == 2) {
                    // the bisector decides (set up above), ties to the smaller label
                    const long long* co = reinterpret_cast<const long long*>(kk + 4);
                    const int i1 = kk[2], i2 = kk[3];
                    const int itie = i1 < i2 ? i1 : i2;
                    const long long step = co[2];
                    long long dv = co[0] + co[1] * c + step * rb;
#pragma unroll
                    for (int k = 0; k < SPL; ++k) {
                        o[k] = dv < 0 ? i1 : (dv > 0 ? i2 : itie);
                        dv += step;
                    }
                } else if (nk <= KMAX) {
                    const float sxf = int_to_f(Q * sx);
                    float syf[SPL];
                    unsigned f1[SPL], f2[SPL];
#pragma unroll
                    for (int k = 0; k < SPL; ++k) {
                        f1[k] = 0x7f800000u;
                        f2[k] = 0x7f800000u;
                        syf[k] = int_to_f(Q * (pyo + rb + k));
                    }
                    for (int j = 0; j < nk; ++j) {
                        const int e = kk[j];
                        const float2 ce = cfs[e];
                        const float dx = sxf - ce.x;
                        const float cyf = ce.y;
                        const float dx2 = dx * dx;
#pragma unroll
                        for (int k = 0; k < SPL; ++k) {
                            const float dy = syf[k] - cyf;
                            const unsigned pk = (__float_as_uint(fmaf(dy, dy, dx2)) & ~63u) | (unsigned)j;
                            const unsigned hi = max(f1[k], pk);
                            f1[k] = min(f1[k], pk);
                            f2[k] = min(f2[k], hi);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < SPL; ++k) {
                        const float a1 = __uint_as_float(f1[k] & ~63u), a2 = __uint_as_float(f2[k] & ~63u);
                        // distances carry 2^-23 rounding and 2^-17 truncation: a gap
                        // above 2^-15 relative means the order is the exact order
                        if (f2[k] == 0x7f800000u || a2 - a1 > a2 * 3.0517578125e-05f)
                            o[k] = ids[kk[f1[k] & 63u]];
                        else
                            o[k] = owner_exact((long long)Q * sx, (long long)Q * (pyo + rb + k), cfs, ids, kk, nk);
                    }
                } else {
                    // more kept centres than the list holds: exact over all scanned
#pragma unroll
                    for (int k = 0; k < SPL; ++k) {
                        const long long qx = (long long)Q * sx, qy = (long long)Q * (pyo + rb + k);
                        long long best = LLONG_MAX;
                        int bi = -1;
                        for (int j = 0; j < n; ++j) {
                            const long long dx = qx - list_int(cfs[j].x), dy = qy - list_int(cfs[j].y);
                            const long long d2 = dx * dx + dy * dy;
                            if (d2 < best || (d2 == best && ids[j] < bi)) { best = d2; bi = ids[j]; }
                        }
                        o[k] = bi;
                    }
                }
#pragma unroll
                for (int k = 0; k < SPL; ++k)
                    if (rb + k < ph && vd_in(P, CHK_OWNER, (long long)(y0 + pyo + rb + k) * Lx + x0 + sx,
                                             (long long)Lx * Ly))
                        ownT[(pyo + rb + k) * Lx + sx] = o[k];
            }
        }
    } else {
        // ---- general path: per-site minimum image, exact int64, over the
        // scanned buckets (the list holds rounded values for far centres) ----
        for (int k = lane; k < ncols * nrows; k += 32) {
            const int lx = k % ncols, ly = k / ncols;
            long long best = LLONG_MAX;
            int bi = -1;
            {
                const long long sx = (long long)Q * (x0 + lx), sy = (long long)Q * (y0 + ly);
                for (int rv = ry0; rv <= ry1; ++rv) {
                    const int rm = rv < 0 ? rv + nby : (rv >= nby ? rv - nby : rv);
                    for (int cu = rx0; cu <= rx1; ++cu) {
                        const int cm = cu < 0 ? cu + nbx : (cu >= nbx ? cu - nbx : cu);
                        const int bk = rm * nbx + cm;
                        for (int j = boff[bk]; j < boff[bk + 1]; ++j) {
                            const int2 cc = bcq[j];
                            const long long dx = wrapM(sx - cc.x, MX), dy = wrapM(sy - cc.y, MY);
                            const long long d2 = dx * dx + dy * dy;
                            const int id = bid[j];
                            if (d2 < best || (d2 == best && id < bi)) { best = d2; bi = id; }
                        }
                    }
                }
            }
            own[(long long)(y0 + ly) * Lx + x0 + lx] = bi;
        }
    }
}

// ---------------------------------------------------------------------------
// Links from the owner array (Section 3.2.2). One warp per 32 x 32 tile. The
// tile's owners plus one row below and one column right (periodic) are
// staged in shared memory with cp.async; the warp then walks the rows, lane l
// at column l.
//
// The tile answers for the adjacencies anchored in it: H(l,r) between sites
// (l,r),(l+1,r) and V(l,r) between (l,r),(l,r+1). Ordering anchors by (row,
// column) with H before V at the same anchor, an adjacency is emitted only if
// none of the earlier adjacencies that share a dual corner with it joins the
// same two owners:
//   H(l,r): H(l,r-1), V(l,r-1), V(l+1,r-1)   (r > 0)
//   V(l,r): H(l-1,r), V(l-1,r) (l > 0), H(l,r)
// Every suppressed adjacency points to a strictly earlier one with the same
// owner pair, which is emitted or suppressed in turn, so by induction over
// the order every pair that meets somewhere is emitted at least once (the
// tiles of the referenced anchors process them). A straight boundary crossing
// the tile is emitted once instead of once per row. Four-owner plaquettes add
// their incircle link. Emitted keys are collected in a per-warp list and
// appended to the instance's link list after merging equal keys.
// ---------------------------------------------------------------------------
constexpr int LINK_WARPS = 4;
constexpr int LSET = 256;       // per-warp key list of the vertex-rule kernel
constexpr int LSET_ADJ = 128;   // per-warp key list of k_links (further keys go straight to the link hash)
constexpr int LS = VW + 4;      // staged row stride (rows start on 16 bytes)

// list entry `pos` of a warp's keys: the link {a, b}, or EMPTY_KEY when an
// end is not a label (obstacle, beyond a wall); past the list, straight into
// the link hash
template <int CAP = LSET>
__device__ __forceinline__ void link_list_put(unsigned long long* list, int pos, int a, int b, const Pools& P,
                                              const InstDesc& D, int inst) {
    const bool ok = (a | b) >= 0;
    if (!vd_in(P, CHK_LINK_LIST, pos, 1ll << 30)) return;
    if (pos < CAP) list[pos] = ok ? edge_key(a, b) : EMPTY_KEY;
    else if (ok) edge_global_insert(P, D, inst, edge_key(a, b));
}

// the first min(n, CAP) keys of a warp's list (whole warp): equal keys within
// a round of 32 are merged, the rest appended to the instance's link list (the
// link hash removes the remaining repeats); EMPTY_KEY entries are dropped
template <int CAP = LSET>
__device__ __forceinline__ void flush_link_list(const unsigned long long* list, int n, int lane, const Pools& P,
                                                const InstDesc& D, int inst) {
    const unsigned lt = (1u << lane) - 1u;
    n = min(n, CAP);
    for (int kb = 0; kb < n; kb += 32) {
        const bool in = kb + lane < n;
        const unsigned long long key = in ? list[kb + lane] : EMPTY_KEY;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const bool has = in && key != EMPTY_KEY && lane == __ffs(grp) - 1;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        if (!m) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(&P.st[inst].n_eapp, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (has) {
            const int pos = base + __popc(m & lt);
            if (pos < D.edge_cap && vd_in(P, CHK_EDGE_APPEND, pos, D.edge_cap)) P.ekeys[D.edge_off + pos] = key;
            else edge_global_insert(P, D, inst, key);   // list full: insert directly
        }
    }
}

__device__ __forceinline__ void cp_async4(int* smem, const int* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(int* smem, const int* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Two phases per tile. 1: lane l walks its column down the rows with the
// owners of the site, its right neighbour and the two below in registers and
// marks the rows where the site differs from its right or lower neighbour
// (about one site in five on Voronoi cells tens of sites wide); 2: the marked
// (row, column) items are compacted into a shared queue and processed with
// every lane on a different item, so the emission rules run with all lanes
// busy instead of with the one or two lanes of a row that cross a boundary.
constexpr int LQ = VW * VH / 2; // queue of marked sites (row * 32 + column) of half a tile

__global__ __launch_bounds__(32 * LINK_WARPS, 8) void k_links(Pools P, StepTable T) {
    pdl_enter();
    __shared__ __align__(16) int s_own[LINK_WARPS][(VH + 1) * LS];
    __shared__ unsigned long long s_list[LINK_WARPS][LSET_ADJ];
    __shared__ unsigned short s_q[LINK_WARPS][LQ];
    __shared__ int s_n[LINK_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * LINK_WARPS + warp;
    if (b >= T.tileV_pre[T.n_act]) return;
    const int a = warp_seg_of_int(T.tileV_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const int K = min(P.st[inst].K, D.comp_cap);
    if (K < 2 || D.edge_rule) return;   // the vertex rule has its own kernel
    const int t = b - T.tileV_pre[a];
    const int tx = t % D.vtx, ty = t / D.vtx;
    const int x0 = tx * VW, y0 = ty * VH;
    const int ncols = min(VW, D.Lx - x0), nrows = min(VH, D.Ly - y0);
    const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
    const int2* cq = P.cq[P.st[inst].slot ^ 1] + D.comp_off;
    const int* own = P.owners + D.site_off;
    int* S = s_own[warp];
    unsigned long long* list = s_list[warp];
    unsigned short* q = s_q[warp];

    // stage rows y0..y0+nrows and columns x0..x0+ncols (both periodic); a
    // full-width tile whose rows start on 16-byte boundaries copies 16 bytes
    // per lane (8 lanes per row), the extra column and other tiles 4 bytes
    const bool vec = ncols == VW && ((D.site_off | D.Lx) & 3) == 0;
    if (vec) {
        const int c4 = (lane & 7) * 4;
        for (int r = lane >> 3; r <= nrows; r += 4) {
            const int y = (y0 + r == D.Ly) ? 0 : y0 + r;
            cp_async16(S + r * LS + c4, own + (long long)y * D.Lx + x0 + c4);
        }
        const int xe = (x0 + VW == D.Lx) ? 0 : x0 + VW;
        for (int r = lane; r <= nrows; r += 32) {
            const int y = (y0 + r == D.Ly) ? 0 : y0 + r;
            cp_async4(S + r * LS + VW, own + (long long)y * D.Lx + xe);
        }
    } else {
        for (int r = 0; r <= nrows; ++r) {
            const int y = (y0 + r == D.Ly) ? 0 : y0 + r;
            const int* row = own + (long long)y * D.Lx;
            for (int c = lane; c <= ncols; c += 32) {
                const int x = (x0 + c == D.Lx) ? 0 : x0 + c;
                cp_async4(S + r * LS + c, row + x);
            }
        }
    }
    if (lane == 0) s_n[warp] = 0;
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();

    // ---- 1. mark the rows where this column's site differs from its right
    // or lower neighbour (only those can anchor an emitted link) ----
    unsigned mark = 0;
    if (lane < ncols) {
        int o = S[lane], rt = S[lane + 1];
        for (int r = 0; r < nrows; ++r) {
            const int dn = S[(r + 1) * LS + lane];
            const int dg = S[(r + 1) * LS + lane + 1];
            mark |= (unsigned)((o != rt) | (o != dn)) << r;
            o = dn;
            rt = dg;
        }
    }
    // the marked sites of rows 0-15, then of rows 16-31, are compacted into
    // the queue (row-major order is not needed) and processed
    for (int h = 0; h < 2; ++h) {
        const unsigned hmark = mark & (h ? 0xffff0000u : 0x0000ffffu);
        const int cnt = __popc(hmark);
        int inc = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += v;
        }
        const int nq = __shfl_sync(0xffffffffu, inc, 31);
        {
            int pos = inc - cnt;
            unsigned m = hmark;
            while (m) {
                const int r = __ffs(m) - 1;
                m &= m - 1;
                if (vd_in(P, CHK_LINK_QUEUE, pos, LQ)) q[pos] = (unsigned short)(r * 32 + lane);
                ++pos;
            }
        }
        __syncwarp();

        // ---- 2. the emission rules at every marked site, one site per lane.
        // The tile answers for the adjacencies anchored in it, H(l,r) between
        // sites (l,r),(l+1,r) and V(l,r) between (l,r),(l,r+1). Ordering anchors
        // by (row, column) with H before V at the same anchor, an adjacency is
        // emitted only if none of the earlier adjacencies that share a dual
        // corner with it joins the same two owners:
        //   H(l,r): H(l,r-1), V(l,r-1), V(l+1,r-1)   (r > 0)
        //   V(l,r): H(l-1,r), V(l-1,r) (l > 0), H(l,r)
        // Every suppressed adjacency points to a strictly earlier one with the
        // same owner pair, which is emitted or suppressed in turn, so by induction
        // over the order every pair that meets somewhere is emitted at least once
        // (the tiles of the referenced anchors process them). A straight boundary
        // crossing the tile is emitted once instead of once per row. Four-owner
        // plaquettes add their incircle link. A pair with a negative owner
        // (obstacle, beyond a wall) is dropped when its key is listed, a plaquette
        // with one before its centres are read.
        for (int i = lane; i < nq; i += 32) {
            const int it = q[i];
            const int r = it >> 5, l = it & 31;
            const int* row = S + r * LS + l;
            const int o = row[0], rt = row[1], dn = row[LS], dg = row[LS + 1];
            if (o != rt) {
                bool sup = false;
                if (r > 0) {
                    const int up = row[-LS], upr = row[-LS + 1];
                    sup = up == rt || upr == o || (up == o && upr == rt);
                }
                if (!sup) link_list_put<LSET_ADJ>(list, atomicAdd(&s_n[warp], 1), o, rt, P, D, inst);
            }
            if (o != dn && rt != dn) {
                bool sup = false;
                if (l > 0) {
                    const int lf = row[-1], dlf = row[LS - 1];
                    sup = lf == dn || (lf == o && dlf == dn);
                }
                if (!sup) link_list_put<LSET_ADJ>(list, atomicAdd(&s_n[warp], 1), o, dn, P, D, inst);
            }
            if (o != rt && o != dn && o != dg && rt != dn && rt != dg && dn != dg) {
                int pa = -1, pb = -1;
                if ((o | rt | dn | dg) >= 0) {
                    const unsigned long long pk = plaquette_key(o, rt, dg, dn, cq, MX, MY);
                    pa = (int)(pk >> 32);
                    pb = (int)(pk & 0xffffffffu);
                }
                link_list_put<LSET_ADJ>(list, atomicAdd(&s_n[warp], 1), pa, pb, P, D, inst);
            }
        }
        __syncwarp();   // the next half overwrites the queue
    }
    __syncwarp();
    flush_link_list<LSET_ADJ>(list, s_n[warp], lane, P, D, inst);
}

// appended links -> link hash (+ degrees); appended pairs -> overlap hash

// which: bit 0 the appended links, bit 1 the appended overlap pairs
__global__ void k_merge_lists(Pools P, StepTable T, int which) {
    pdl_enter();
    __shared__ long long s_pe[SEG_CACHE], s_po[SEG_CACHE];
    __shared__ int s_act[SEG_CACHE];
    const int* act;
    const long long* pe = seg_table(pre_arr(T, PRE_EA), T.act, T.n_act, s_pe, s_act, &act);
    const long long* po = seg_table(pre_arr(T, PRE_OA), T.n_act, s_po);
    const long long ne = (which & 1) ? pe[T.n_act] : 0, no = (which & 2) ? po[T.n_act] : 0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ne + no;
         g += (long long)gridDim.x * blockDim.x) {
        if (g < ne) {
            const int a = seg_of(pe, T.n_act, g);
            const int inst = act[a];
            const InstDesc& D = P.desc[inst];
            edge_global_insert(P, D, inst, P.ekeys[D.edge_off + (g - pe[a])]);
        } else {
            const long long h = g - ne;
            const int a = seg_of(po, T.n_act, h);
            const int inst = act[a];
            const InstDesc& D = P.desc[inst];
            const long long j = D.ovl_off + (h - po[a]);
            ovl_global_insert(P, D, inst, P.oapp_key[j], P.oapp_cnt[j]);
        }
    }
}

void launch_merge_lists(const Launch& L) {
    launch_plan(L, 0, ENDS_NONE);
    launch_step(L, k_merge_lists, dim3(L.grid_wide), dim3(256), L.P, L.T, 3);
}

void launch_merge_edges(const Launch& L) {
    launch_plan(L, 0, ENDS_NONE, pre_bit(PRE_EA));
    launch_step(L, k_merge_lists, dim3(L.grid_wide), dim3(256), L.P, L.T, 1);
}

void launch_merge_overlaps(const Launch& L) {
    launch_plan(L, 0, ENDS_NONE, pre_bit(PRE_OA));
    launch_step(L, k_merge_lists, dim3(L.grid_wide), dim3(256), L.P, L.T, 2);
}

void launch_voronoi(const Launch& L) {
    const dim3 grid((L.total_tilesA + VWARPS - 1) / VWARPS), block(32 * VWARPS);
    switch (L.vpatch) {
        case VPATCH_16x8: launch_step(L, k_voronoi<16, 8>, grid, block, L.P, L.T); break;
        case VPATCH_32x8: launch_step(L, k_voronoi<32, 8>, grid, block, L.P, L.T); break;
        case VPATCH_16x16: launch_step(L, k_voronoi<16, 16>, grid, block, L.P, L.T); break;
        default: launch_step(L, k_voronoi<8, 8>, grid, block, L.P, L.T); break;
    }
}

// ---------------------------------------------------------------------------
// The paper's link rule (Section 3.2.2), an option: links are read only at
// vertex sites, i.e. sites with three or more colour changes around their
// 8-site frame. With e1 one of +x, +y, -x, -y and e2 = e1 turned a quarter
// counter-clockwise, the conditions written for spx and spxpy apply to the
// four quarter turns:
//   first neighbour k+e1: C(k+e1) != C(k) and C(k+e2) != C(k+e1-e2);
//   second neighbour k+e1+e2: C(k+e1+e2) != C(k), C(k+e2) != C(k+e1-e2),
//   C(k+e2) != C(k+e1), and the inner-frame point (read as the plaquette
//   centre k + (e1+e2)/2) is owned by C(k) or by C(k+e1+e2).
// One warp per 32 x 32 tile, lane = column: the tile's owners with a one-site
// halo are staged in shared memory with cp.async (all rows in flight at once),
// then the warp walks down the rows with the rows above and below in
// registers. Vertex sites are rare: a row without one skips the rules. The
// colour of a plaquette centre is its Voronoi colour, the nearest centre over
// all centres (exact, ties to the smallest label), found by a ring search of
// the frame's bucket grid that starts from the nearest corner colour. Keys go
// to the per-warp list, merged and appended as in the adjacency rule.
// ---------------------------------------------------------------------------

// Voronoi colour of the point (qx, qy) (1/1024 site, in [0, MX) x [0, MY)):
// the nearest centre over all centres, exact int64 minimum-image distances,
// ties to the smallest label. (best, bd) is a centre already known and its
// squared distance, so every centre that can win or tie lies within
// rho = ceil(sqrt(bd)) of the point on each axis; the buckets overlapping that
// square (at most two runs of bucket columns and rows, split where the square
// wraps around the lattice) hold all of them. Centres and the point both lie
// in [0, M), so one conditional step gives the minimum image.
__device__ __forceinline__ long long isqrt_ceil(long long v) {
    long long r = (long long)ceil(sqrt((double)v));
    while (r > 0 && (r - 1) * (r - 1) >= v) --r;
    while (r * r < v) ++r;
    return r;
}

// site interval [lo, hi] (unwrapped, hi - lo < L) as at most two runs of
// bucket indices on a ring of L sites cut into buckets of B (the last one
// possibly narrower)
__device__ __forceinline__ int bucket_runs(long long lo, long long hi, int L, int B, int nb, int* b0, int* b1) {
    if (hi - lo + 1 >= L) {
        b0[0] = 0;
        b1[0] = nb - 1;
        return 1;
    }
    long long a = lo % L;
    if (a < 0) a += L;
    const long long e = a + (hi - lo);
    if (e < L) {
        b0[0] = (int)(a / B);
        b1[0] = (int)(e / B);
        return 1;
    }
    b0[0] = (int)(a / B);
    b1[0] = nb - 1;
    b0[1] = 0;
    b1[1] = (int)((e - L) / B);
    return 2;
}

__device__ int point_owner(const int* boff, const int2* bcq, const int* bid, int B, int nbx, int nby, long long qx,
                           long long qy, int Lx, int Ly, int best, long long bd) {
    const long long MX = (long long)Q * Lx, MY = (long long)Q * Ly, HX = MX >> 1, HY = MY >> 1;
    const long long rho = isqrt_ceil(bd);
    int cx0[2], cx1[2], cy0[2], cy1[2];
    const int nxr = bucket_runs((qx - rho) >> 10, (qx + rho) >> 10, Lx, B, nbx, cx0, cx1);
    const int nyr = bucket_runs((qy - rho) >> 10, (qy + rho) >> 10, Ly, B, nby, cy0, cy1);
    for (int ry = 0; ry < nyr; ++ry)
        for (int rv = cy0[ry]; rv <= cy1[ry]; ++rv)
            for (int rx = 0; rx < nxr; ++rx)
                for (int cu = cx0[rx]; cu <= cx1[rx]; ++cu) {
                    const int bk = rv * nbx + cu;
                    for (int j = boff[bk]; j < boff[bk + 1]; ++j) {
                        const int2 c = bcq[j];
                        long long ddx = (long long)c.x - qx + HX, ddy = (long long)c.y - qy + HY;
                        ddx = (ddx < 0 ? ddx + MX : (ddx >= MX ? ddx - MX : ddx)) - HX;
                        ddy = (ddy < 0 ? ddy + MY : (ddy >= MY ? ddy - MY : ddy)) - HY;
                        const long long d = ddx * ddx + ddy * ddy;
                        const int id = bid[j];
                        if (d < bd || (d == bd && id < best)) {
                            bd = d;
                            best = id;
                        }
                    }
                }
    return best;
}

// v mod L for -L <= v < 2L, without a division (a 64-bit remainder is a long
// dependent chain, and vertex sites take it one lane at a time): plaquette
// centres lie within half a site of the lattice and centres are stored in
// [0, Q L), so their differences stay in range
__device__ __forceinline__ long long wrap_once(long long v, long long L) {
    return v < 0 ? v + L : (v >= L ? v - L : v);
}

constexpr int VS = VW + 8;      // staged row stride of the vertex rule: column c at 4 + c
constexpr int VQ = 256;         // queued plaquette-centre searches per warp

__global__ __launch_bounds__(32 * LINK_WARPS) void k_links_vertex(Pools P, StepTable T) {
    pdl_enter();
    __shared__ __align__(16) int s_own[LINK_WARPS][(VH + 2) * VS];
    __shared__ unsigned long long s_list[LINK_WARPS][LSET];
    // plaquette centres whose colour needs the search: (k, diagonal colour,
    // best corner colour, site, quarter turn), resolved with every lane busy
    __shared__ int s_q[LINK_WARPS][VQ][4];
    __shared__ int s_qn[LINK_WARPS], s_ln[LINK_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * LINK_WARPS + warp;
    if (b >= T.tileV_pre[T.n_act]) return;
    const int a = warp_seg_of_int(T.tileV_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const InstState& St = P.st[inst];
    const int K = min(St.K, D.comp_cap);
    if (K < 2 || !D.edge_rule) return;
    const int t = b - T.tileV_pre[a];
    const int tx = t % D.vtx, ty = t / D.vtx;
    const int Lx = D.Lx, Ly = D.Ly;
    const int x0 = tx * VW, y0 = ty * VH;
    const int ncols = min(VW, Lx - x0), nrows = min(VH, Ly - y0);
    const int2* cq = P.cq[St.slot ^ 1] + D.comp_off;
    const int* boff = P.boff[St.slot ^ 1] + D.bucket_off;
    const int2* bcq = P.bcq[St.slot ^ 1] + D.comp_off;
    const int* bid = P.bid[St.slot ^ 1] + D.comp_off;
    const int* own = P.owners + D.site_off;
    const long long MX = (long long)Q * Lx, MY = (long long)Q * Ly, HX = MX / 2, HY = MY / 2;
    int* S = s_own[warp];
    unsigned long long* list = s_list[warp];
    if (lane == 0) s_qn[warp] = 0;

    // stage rows y0-1 .. y0+nrows and columns x0-1 .. x0+ncols (both periodic):
    // staged row r holds lattice row y0-1+r, column c lattice column x0+c at
    // S[r * VS + 4 + c]; a full-width tile whose rows start on 16-byte
    // boundaries copies its 32 columns 16 bytes per lane, the halo 4 bytes
    auto wrap_row = [&](int y) { return y < 0 ? y + Ly : (y >= Ly ? y - Ly : y); };
    const bool vec = ncols == VW && ((D.site_off | Lx) & 3) == 0;
    if (vec) {
        const int c4 = (lane & 7) * 4;
        for (int r = lane >> 3; r < nrows + 2; r += 4)
            cp_async16(S + r * VS + 4 + c4, own + (long long)wrap_row(y0 - 1 + r) * Lx + x0 + c4);
        const int xl = x0 == 0 ? Lx - 1 : x0 - 1, xr = x0 + VW == Lx ? 0 : x0 + VW;
        for (int r = lane; r < nrows + 2; r += 32) {
            const int* row = own + (long long)wrap_row(y0 - 1 + r) * Lx;
            cp_async4(S + r * VS + 3, row + xl);
            cp_async4(S + r * VS + 4 + VW, row + xr);
        }
    } else {
        for (int r = 0; r < nrows + 2; ++r) {
            const int* row = own + (long long)wrap_row(y0 - 1 + r) * Lx;
            for (int c = lane - 1; c <= ncols; c += 32) {
                const int xx = x0 + c < 0 ? x0 + c + Lx : (x0 + c >= Lx ? x0 + c - Lx : x0 + c);
                cp_async4(S + r * VS + 4 + c, row + xx);
            }
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();

    // lanes past the last column read the last column and emit nothing
    const bool valid = lane < ncols;
    const int x = x0 + lane;
    const int* sc = S + 4 + min(lane, ncols - 1);
    // rows y-1 and y in registers (columns x-1, x, x+1), row y+1 read per step
    int um = sc[-1], u0 = sc[0], up = sc[1];
    int om = sc[VS - 1], o0 = sc[VS], op = sc[VS + 1];
    int n = 0;   // keys in the warp's list (warp-uniform)
    // the queued plaquette centres: colour by search, link when it is k's or
    // the diagonal neighbour's (whole warp; n is updated)
    auto resolve = [&]() {
        __syncwarp();
        const int nq = s_qn[warp];
        if (lane == 0) s_ln[warp] = n;
        __syncwarp();
        for (int i2 = lane; i2 < nq; i2 += 32) {
            const int* it = s_q[warp][i2];
            const int k = it[0], cd = it[1], ca0 = it[2], site = it[3] >> 2, q = it[3] & 3;
            const int yy = site / Lx, xx = site - yy * Lx;
            const int ex = (q == 0 || q == 3) ? 1 : -1, ey = (q == 0 || q == 1) ? 1 : -1;
            const long long qx = wrap_once((long long)Q * xx + (Q / 2) * ex, MX);
            const long long qy = wrap_once((long long)Q * yy + (Q / 2) * ey, MY);
            const int2 cc = cq[ca0];
            const long long ddx = wrap_once((long long)cc.x - qx + HX, MX) - HX;
            const long long ddy = wrap_once((long long)cc.y - qy + HY, MY) - HY;
            const int ca = point_owner(boff, bcq, bid, St.B, St.nbx, St.nby, qx, qy, Lx, Ly, ca0,
                                       ddx * ddx + ddy * ddy);
            if (ca == k || ca == cd) link_list_put(list, atomicAdd(&s_ln[warp], 1), k, cd, P, D, inst);
        }
        __syncwarp();
        n = s_ln[warp];
        if (lane == 0) s_qn[warp] = 0;
        __syncwarp();
    };
    for (int ri = 0; ri < nrows; ++ri) {
        __syncwarp();   // the queue count is read by every lane alike
        if (s_qn[warp] > VQ - 4 * 32) resolve();   // a row adds at most 4 items per lane
        const int y = y0 + ri;
        const int* sd = sc + (ri + 2) * VS;
        const int dm = sd[-1], d0 = sd[0], dp = sd[1];
        // the frame in counter-clockwise order from +x; f[8] = the site itself
        int f[9];
        f[0] = op; f[1] = dp; f[2] = d0; f[3] = dm;
        f[4] = om; f[5] = um; f[6] = u0; f[7] = up;
        f[8] = o0;
        // colour changes around the frame; members beyond a wall (owner
        // OWN_OUTSIDE) leave it, obstacles keep their MAXLINK colour
        int prev = OWN_OUTSIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) prev = f[i] != OWN_OUTSIDE ? f[i] : prev;
        int gaps = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (f[i] != OWN_OUTSIDE) {
                gaps += f[i] != prev ? 1 : 0;
                prev = f[i];
            }
        const int k = f[8];
        const bool vert = valid && gaps >= 3 && k >= 0;
        if (__any_sync(0xffffffffu, vert)) {
            // bit q: first neighbour of quarter turn q; bit 4 + q: second neighbour
            unsigned em = 0;
            if (vert) {
                // quarter turn q: e1 = frame entry 2q, e1 + e2 = entry 2q + 1,
                // e2 = entry 2q + 2, e1 - e2 = entry 2q - 1 (all mod 8)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c1 = f[2 * q], cd = f[2 * q + 1], c2 = f[(2 * q + 2) & 7], c3 = f[(2 * q + 7) & 7];
                    if (c1 >= 0 && c1 != k && c2 != c3) em |= 1u << q;
                    if (cd >= 0 && cd != k && c2 != c3 && c2 != c1) {
                        // plaquette centre k + (e1 + e2) / 2: its Voronoi colour,
                        // searched from the nearest of the corner colours k, k+e1,
                        // k+e1+e2, k+e2
                        const int ex = (q == 0 || q == 3) ? 1 : -1, ey = (q == 0 || q == 1) ? 1 : -1;
                        long long qx = (long long)Q * x + (Q / 2) * ex, qy = (long long)Q * y + (Q / 2) * ey;
                        qx = wrap_once(qx, MX);
                        qy = wrap_once(qy, MY);
                        const int cand[4] = {k, c1, cd, c2};
                        int ca = -1;
                        long long bd = 0;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int c = cand[j];
                            if (c < 0) continue;
                            const int2 cc = cq[c];
                            const long long ddx = wrap_once((long long)cc.x - qx + HX, MX) - HX;
                            const long long ddy = wrap_once((long long)cc.y - qy + HY, MY) - HY;
                            const long long d = ddx * ddx + ddy * ddy;
                            if (ca < 0 || d < bd || (d == bd && c < ca)) {
                                bd = d;
                                ca = c;
                            }
                        }
                        // a centre that owns no corner can only take the point
                        // from a corner colour; when that colour is neither end
                        // of the diagonal the answer is no link either way, else
                        // the point is queued for the search
                        if (ca == k || ca == cd) {
                            int* it = s_q[warp][atomicAdd(&s_qn[warp], 1)];
                            it[0] = k;
                            it[1] = cd;
                            it[2] = ca;
                            it[3] = ((y * Lx + x) << 2) | q;
                        }
                    }
                }
            }
            // this lane's keys go after those of the lanes before it
            const int ne = __popc(em);
            int inc = ne;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += v;
            }
            int pos = n + inc - ne;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (em & (1u << q)) link_list_put(list, pos++, k, f[2 * q], P, D, inst);
                if (em & (16u << q)) link_list_put(list, pos++, k, f[2 * q + 1], P, D, inst);
            }
            n += __shfl_sync(0xffffffffu, inc, 31);
        }
        um = om; u0 = o0; up = op;
        om = dm; o0 = d0; op = dp;
    }
    resolve();
    flush_link_list(list, n, lane, P, D, inst);
}

// Owners of sites beyond a wall (the second half of a bounded axis) become
// OWN_OUTSIDE and owners of obstacle sites OWN_OBSTACLE (the paper's MAXLINK
// colour), so that no link is read there; one warp per 32 x 32 tile.
__global__ __launch_bounds__(32 * LINK_WARPS) void k_mask_owners(Pools P, StepTable T) {
    pdl_enter();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * LINK_WARPS + warp;
    if (b >= T.tileV_pre[T.n_act]) return;
    const int a = warp_seg_of_int(T.tileV_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    if (!D.masked) return;
    const int t = b - T.tileV_pre[a];
    const int tx = t % D.vtx, ty = t / D.vtx;
    const int x = tx * VW + lane;
    if (x >= D.Lx) return;
    int* own = P.owners + D.site_off;
    const unsigned* ob = P.obst + D.word_off;
    for (int y = ty * VH; y < min(ty * VH + VH, D.Ly); ++y) {
        int* o = own + (long long)y * D.Lx + x;
        if (x >= D.uLx || y >= D.uLy) *o = OWN_OUTSIDE;
        else if ((ob[(long long)y * D.wpr + (x >> 5)] >> (x & 31)) & 1u) *o = OWN_OBSTACLE;
    }
}

// k_links holds 35 KB of shared memory per block; six blocks per SM (the
// register bound of its launch bounds) need the largest shared-memory
// carveout, which the driver need not choose by itself. Host-side, once per
// context creation, outside any stream capture.
void set_kernel_attributes() {
    if (cudaFuncSetAttribute(k_links, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        cudaGetLastError();   // a preference only: the kernel runs either way
}

void launch_links(const Launch& L) {
    if (L.masked)
        launch_step(L, k_mask_owners, dim3((L.total_tilesV + LINK_WARPS - 1) / LINK_WARPS), dim3(32 * LINK_WARPS),
                    L.P, L.T);
    launch_step(L, k_links, dim3((L.total_tilesV + LINK_WARPS - 1) / LINK_WARPS), dim3(32 * LINK_WARPS), L.P, L.T);
    if (L.vertex_rule)
        launch_step(L, k_links_vertex, dim3((L.total_tilesV + LINK_WARPS - 1) / LINK_WARPS), dim3(32 * LINK_WARPS),
                    L.P, L.T);
}

}  // namespace vd
