// Digital Voronoi colouring (Section 3.2.1) and Delaunay links (Section 3.2.2).
//
// owner(s) = argmin_i |1024*s - c_i|^2 over all bubble centres (exact int64,
// minimum image on the torus, ties to the smallest label). The paper computes
// this by scanning every centre from every site; here each 32 x 32 tile first
// collects a provably complete candidate set from a bucket grid of centres:
//   U     = min over scanned centres of an upper bound of their largest
//           distance to the tile (so every site has a centre within U),
//   keep  = centres whose smallest distance to the tile is <= U,
// scanning rings of buckets around the tile until the unscanned region is
// farther than sqrt(U). Each site then scans only the kept candidates.
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
            if (idx < D.edge_cap) P.elist[D.edge_off + idx] = (int)h;
            else atomicOr(&P.st[inst].err, ERR_EDGE_CAP);
            atomicAdd(&P.deg[D.comp_off + (int)(key >> 32)], 1);
            return;
        }
        if (k == key) return;
        h = (h + 1) & mask;
    }
    atomicOr(&P.st[inst].err, ERR_EDGE_CAP);
}


constexpr int WCAND = 64;   // per-warp candidate list

// Exact owner over a candidate list with int64 distances (rel. coordinates,
// no wrap needed), ties to the smallest label.
__device__ __forceinline__ int owner_exact(long long sx, long long sy, const int* cx, const int* cy, const int* id,
                                           int n) {
    long long best = LLONG_MAX;
    int bi = -1;
    for (int j = 0; j < n; ++j) {
        const long long dx = sx - cx[j], dy = sy - cy[j];
        const long long d2 = dx * dx + dy * dy;
        if (d2 < best || (d2 == best && id[j] < bi)) { best = d2; bi = id[j]; }
    }
    return bi;
}

__global__ __launch_bounds__(VTHREADS) void k_voronoi(Pools P, StepTable T) {
    // centres scanned by the ring search, relative to the tile origin (minimum image)
    __shared__ int s_cx[VCAND], s_cy[VCAND], s_id[VCAND];
    // per-warp candidate lists of each warp's 16 x 8 patch
    __shared__ float s_wfx[8][WCAND], s_wfy[8][WCAND];
    __shared__ int s_wix[8][WCAND], s_wiy[8][WCAND], s_wid[8][WCAND];
    __shared__ int s_own[VH][VW + 1];
    __shared__ int s_n, s_over;
    __shared__ unsigned long long s_U;

    const int b = blockIdx.x;
    const int a = seg_of_int(T.tileV_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileV_pre[a];
    const int tx = t % D.vtx, ty = t / D.vtx;
    const int x0 = tx * VW, y0 = ty * VH;
    const int ncols = min(VW, D.Lx - x0), nrows = min(VH, D.Ly - y0);
    const int K = min(S.K, D.comp_cap);
    const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
    const long long X0 = (long long)Q * x0, Y0 = (long long)Q * y0;
    const long long WR = (long long)Q * (ncols - 1), HR = (long long)Q * (nrows - 1);   // core sites only
    const int2* cq = P.cq + D.comp_off;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        s_n = 0;
        s_over = 0;
        s_U = ULLONG_MAX;
    }
    __syncthreads();

    if (K > 0) {
        // ---- ring search over the bucket grid (all threads) ----
        // Bucket indices are unwrapped (they may run below 0 or past nb-1 by
        // less than one period); all arithmetic is 32-bit here.
        const int Bk = S.B, nbx = S.nbx, nby = S.nby;
        const int bx0 = x0 / Bk, bx1 = (x0 + ncols - 1) / Bk;
        const int by0 = y0 / Bk, by1 = (y0 + nrows - 1) / Bk;
        const int* boff = P.boff + D.bucket_off;
        const int2* bcq = P.bcq + D.comp_off;
        const int* bid = P.bid + D.comp_off;
        int px0 = 0, px1 = -1, py0 = 0, py1 = -1;
        bool pfx = false, pfy = false, have_prev = false;
        unsigned long long myU = ULLONG_MAX;
        // the first round takes rings 0..2 at once (one latency round instead of three)
        for (int r = 2;; ++r) {
            int rx0 = bx0 - r, rx1 = bx1 + r, ry0 = by0 - r, ry1 = by1 + r;
            const bool fx = (rx1 - rx0 + 1) >= nbx, fy = (ry1 - ry0 + 1) >= nby;
            if (fx) { rx0 = 0; rx1 = nbx - 1; }
            if (fy) { ry0 = 0; ry1 = nby - 1; }
            const int wx = rx1 - rx0 + 1, wy = ry1 - ry0 + 1;
            const int ncell = wx * wy;
            for (int kb = warp * 32; kb < ncell; kb += VTHREADS) {   // warp-uniform loop
                const int k = kb + lane;
                int jb = 0, je = 0;
                if (k < ncell) {
                    const int kr = k / wx;
                    const int cu = rx0 + (k - kr * wx), rv = ry0 + kr;
                    bool skip = false;
                    if (have_prev) {
                        int dxp = cu - px0, dyp = rv - py0;
                        if (dxp < 0) dxp += nbx; else if (dxp >= nbx) dxp -= nbx;
                        if (dyp < 0) dyp += nby; else if (dyp >= nby) dyp -= nby;
                        skip = (pfx || dxp <= px1 - px0) && (pfy || dyp <= py1 - py0);
                    }
                    if (!skip) {
                        const int cm = cu < 0 ? cu + nbx : (cu >= nbx ? cu - nbx : cu);
                        const int rm = rv < 0 ? rv + nby : (rv >= nby ? rv - nby : rv);
                        const int bk = rm * nbx + cm;
                        jb = boff[bk];
                        je = boff[bk + 1];
                    }
                }
                // one shared-memory reservation per warp
                const int cnt = je - jb;
                int inc = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                const int tot = __shfl_sync(0xffffffffu, inc, 31);
                int base = 0;
                if (lane == 31 && tot > 0) base = atomicAdd(&s_n, tot);
                base = __shfl_sync(0xffffffffu, base, 31) + inc - cnt;
                for (int j = jb; j < je; ++j, ++base) {
                    const int2 c = bcq[j];
                    const long long ddx = wrapM((long long)c.x - X0, MX);
                    const long long ddy = wrapM((long long)c.y - Y0, MY);
                    long long mxx = max(ddx < 0 ? -ddx : ddx, (ddx - WR) < 0 ? WR - ddx : ddx - WR);
                    long long mxy = max(ddy < 0 ? -ddy : ddy, (ddy - HR) < 0 ? HR - ddy : ddy - HR);
                    mxx = min(mxx, MX >> 1);
                    mxy = min(mxy, MY >> 1);
                    const unsigned long long u = (unsigned long long)(mxx * mxx + mxy * mxy);
                    myU = u < myU ? u : myU;
                    if (base < VCAND) {
                        s_cx[base] = (int)ddx;
                        s_cy[base] = (int)ddy;
                        s_id[base] = bid[j];
                    } else {
                        s_over = 1;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long v = __shfl_xor_sync(0xffffffffu, myU, o);
                myU = v < myU ? v : myU;
            }
            if (lane == 0 && myU != ULLONG_MAX) atomicMin(&s_U, myU);
            __syncthreads();
            if (fx && fy) break;
            // gap between the region and the unscanned buckets (periods handled by
            // one conditional shift: the ranges are narrower than a period here)
            long long g = LLONG_MAX;
            if (!fx) {
                const int lx = rx0 < 0 ? (rx0 + nbx) * Bk - D.Lx : rx0 * Bk;            // start of bucket rx0
                const int ex = rx1 >= nbx ? min((rx1 - nbx + 1) * Bk, D.Lx) + D.Lx      // end of bucket rx1
                                          : min((rx1 + 1) * Bk, D.Lx);
                g = min((long long)Q * (x0 - lx), (long long)Q * (ex - (x0 + ncols - 1)));
            }
            if (!fy) {
                const int ly = ry0 < 0 ? (ry0 + nby) * Bk - D.Ly : ry0 * Bk;
                const int ey = ry1 >= nby ? min((ry1 - nby + 1) * Bk, D.Ly) + D.Ly : min((ry1 + 1) * Bk, D.Ly);
                g = min(g, min((long long)Q * (y0 - ly), (long long)Q * (ey - (y0 + nrows - 1))));
            }
            const unsigned long long U = s_U;
            __syncthreads();
            // every unscanned centre is at least g away from the region
            if (g > 0 && (g >= (1ll << 31) || (unsigned long long)(g * g) > U)) break;
            px0 = rx0; px1 = rx1; py0 = ry0; py1 = ry1; pfx = fx; pfy = fy; have_prev = true;
        }
    }

    // Each warp filters the scanned centres for its own patch; a scanned set
    // holds every centre within U of the tile, so it holds every patch owner.
    const int px0 = (warp & 1) * 16, py0 = (warp >> 1) * 8;
    const int cbx = min(px0 + 15, ncols - 1);
    const int rbx = min(py0 + 7, nrows - 1);
    const bool has_patch = (px0 < ncols) && (py0 < nrows);
    int wn = 0;
    bool wover = false, wbad = false;
    const int nscan = min(s_n, VCAND);
    if (K > 0 && !s_over && has_patch) {
        const long long PX0 = (long long)Q * px0, PY0 = (long long)Q * py0;
        const long long PW = (long long)Q * (cbx - px0), PH = (long long)Q * (rbx - py0);
        long long Uw = LLONG_MAX;
        for (int k = lane; k < nscan; k += 32) {
            const long long dx = s_cx[k] - PX0, dy = s_cy[k] - PY0;
            const long long mxx = max(dx < 0 ? -dx : dx, dx > PW ? dx - PW : PW - dx);
            const long long mxy = max(dy < 0 ? -dy : dy, dy > PH ? dy - PH : PH - dy);
            Uw = min(Uw, mxx * mxx + mxy * mxy);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Uw = min(Uw, __shfl_xor_sync(0xffffffffu, Uw, o));
        for (int base = 0; base < nscan; base += 32) {
            const int k = base + lane;
            bool keep = false;
            if (k < nscan) {
                const int cx = s_cx[k], cy = s_cy[k];
                const long long dx = cx - PX0, dy = cy - PY0;
                const long long ex = dx < 0 ? -dx : (dx > PW ? dx - PW : 0);
                const long long ey = dy < 0 ? -dy : (dy > PH ? dy - PH : 0);
                keep = ex * ex + ey * ey <= Uw;
                // The fast path needs every scanned centre's tile-relative position to
                // be its minimum image for every site of the region (otherwise the
                // distances above are not the torus distances) and exact in float32
                // (|v| < 2^23). Any exception sends the warp to the exact general path.
                if (!((long long)cx > WR - (MX >> 1) && (long long)cy > HR - (MY >> 1) &&
                      cx < (1 << 23) && cx > -(1 << 23) && cy < (1 << 23) && cy > -(1 << 23)))
                    wbad = true;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = wn + __popc(m & ((1u << lane) - 1u));
                if (pos < WCAND) {
                    s_wix[warp][pos] = s_cx[k];
                    s_wiy[warp][pos] = s_cy[k];
                    s_wfx[warp][pos] = (float)s_cx[k];
                    s_wfy[warp][pos] = (float)s_cy[k];
                    s_wid[warp][pos] = s_id[k];
                }
            }
            wn += __popc(m);
        }
        wbad = __any_sync(0xffffffffu, wbad);
        wover = wn > WCAND;
        __syncwarp();
    }

    const bool fast = (K > 0) && !s_over && !wbad;
    if (fast && has_patch) {
        const float* wfx = s_wfx[warp];
        const int n = wover ? nscan : wn;
        // sites: lane -> column px0 + (lane & 15), rows py0 + 4*(lane >> 4) .. +3;
        // then the halo column/row sites outside that 16 x 8 block
        const int c = px0 + (lane & 15);
        const int rb = py0 + 4 * (lane >> 4);
        if (c <= cbx && rb <= rbx) {
            const float sxf = (float)(Q * c);
            float syf[4];
            float f1[4], f2[4];
            int i1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                f1[k] = INFINITY; f2[k] = INFINITY; i1[k] = -1;
                syf[k] = (float)(Q * (rb + k));
            }
            if (!wover) {
                for (int j = 0; j < n; ++j) {
                    const float dx = sxf - wfx[j];
                    const float dx2 = dx * dx;
                    const float fy = s_wfy[warp][j];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float dy = syf[k] - fy;
                        const float d = fmaf(dy, dy, dx2);
                        if (d < f1[k]) { f2[k] = f1[k]; f1[k] = d; i1[k] = j; }
                        else f2[k] = fminf(f2[k], d);
                    }
                }
            } else {
                for (int j = 0; j < n; ++j) {
                    const float dx = sxf - (float)s_cx[j];
                    const float dx2 = dx * dx;
                    const float fy = (float)s_cy[j];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float dy = syf[k] - fy;
                        const float d = fmaf(dy, dy, dx2);
                        if (d < f1[k]) { f2[k] = f1[k]; f1[k] = d; i1[k] = j; }
                        else f2[k] = fminf(f2[k], d);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rr = rb + k;
                if (rr > rbx) break;
                int o;
                // a gap above 2^-20 relative means the float32 order is the exact order
                // (the float32 distance is within 2^-23 relative of the exact one)
                if (f2[k] == INFINITY || f2[k] - f1[k] > f2[k] * 9.5367431640625e-07f) {
                    o = wover ? s_id[i1[k]] : s_wid[warp][i1[k]];
                } else {
                    o = wover ? owner_exact((long long)Q * c, (long long)Q * rr, s_cx, s_cy, s_id, n)
                              : owner_exact((long long)Q * c, (long long)Q * rr, s_wix[warp], s_wiy[warp],
                                            s_wid[warp], n);
                }
                s_own[rr][c] = o;
            }
        }
    } else if (has_patch) {
        // ---- general path for this warp's sites: per-site minimum image over
        // the scanned centres (or over all centres when the scan overflowed) ----
        const bool all = (K > 0) && s_over;
        const int nc = all ? K : (K > 0 ? nscan : 0);
        const int ew = cbx - px0 + 1, eh = rbx - py0 + 1;
        for (int k = lane; k < ew * eh; k += 32) {
            const int lx = px0 + k % ew, ly = py0 + k / ew;
            const long long sx = (long long)Q * lx, sy = (long long)Q * ly;   // relative to the tile origin
            long long best = LLONG_MAX;
            int bi = -1;
            for (int j = 0; j < nc; ++j) {
                long long cx, cy;
                int id;
                if (all) {
                    cx = wrapM((long long)cq[j].x - X0, MX);
                    cy = wrapM((long long)cq[j].y - Y0, MY);
                    id = j;
                } else {
                    cx = s_cx[j]; cy = s_cy[j]; id = s_id[j];
                }
                const long long dx = wrapM(sx - cx, MX), dy = wrapM(sy - cy, MY);
                const long long d2 = dx * dx + dy * dy;
                if (d2 < best || (d2 == best && id < bi)) { best = d2; bi = id; }
            }
            s_own[ly][lx] = bi;
        }
    }
    __syncthreads();

    // ---- write owners of the core tile ----
    int* own = P.owners + D.site_off;
    for (int k = threadIdx.x; k < VW * VH / 4; k += VTHREADS) {
        const int ly = k / (VW / 4), lx = (k % (VW / 4)) * 4;
        if (ly >= nrows || lx >= ncols) continue;
        int* o = own + (long long)(y0 + ly) * D.Lx + x0 + lx;
        if (lx + 4 <= ncols && ((reinterpret_cast<uintptr_t>(o) & 15u) == 0)) {
            *reinterpret_cast<int4*>(o) = make_int4(s_own[ly][lx], s_own[ly][lx + 1], s_own[ly][lx + 2], s_own[ly][lx + 3]);
        } else {
            for (int i = 0; i < 4 && lx + i < ncols; ++i) o[i] = s_own[ly][lx + i];
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
constexpr int LSET = 256;       // per-warp key list
constexpr int LS = VW + 4;      // staged row stride (rows start on 16 bytes)

// slot `pos` of a warp's key list; past its end the key goes to the hash
__device__ __forceinline__ void link_list_put(unsigned long long* list, int pos, unsigned long long key,
                                              const Pools& P, const InstDesc& D, int inst) {
    if (pos < LSET) list[pos] = key;
    else edge_global_insert(P, D, inst, key);
}

__device__ __forceinline__ void cp_async4(int* smem, const int* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(int* smem, const int* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__global__ __launch_bounds__(32 * LINK_WARPS) void k_links(Pools P, StepTable T) {
    __shared__ __align__(16) int s_own[LINK_WARPS][(VH + 1) * LS];
    __shared__ unsigned long long s_list[LINK_WARPS][LSET];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * LINK_WARPS + warp;
    if (b >= T.tileV_pre[T.n_act]) return;
    const int a = seg_of_int(T.tileV_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc& D = P.desc[inst];
    const int K = min(P.st[inst].K, D.comp_cap);
    if (K < 2) return;
    const int t = b - T.tileV_pre[a];
    const int tx = t % D.vtx, ty = t / D.vtx;
    const int x0 = tx * VW, y0 = ty * VH;
    const int ncols = min(VW, D.Lx - x0), nrows = min(VH, D.Ly - y0);
    const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
    const int2* cq = P.cq + D.comp_off;
    const int* own = P.owners + D.site_off;
    int* S = s_own[warp];
    unsigned long long* list = s_list[warp];

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
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();

    const bool valid = lane < ncols;
    const int l = min(lane, ncols - 1);
    const unsigned lt = (1u << lane) - 1u;
    int o = S[l], rt = S[l + 1];
    int up = 0, upr = 0;
    int lf = __shfl_up_sync(0xffffffffu, o, 1);
    int n = 0;   // keys in the warp's list (warp-uniform)
    for (int r = 0; r < nrows; ++r) {
        const int dn = S[(r + 1) * LS + l];
        const int dg = S[(r + 1) * LS + l + 1];
        const int dlf = __shfl_up_sync(0xffffffffu, dn, 1);
        const bool eh = valid && o != rt && !(r > 0 && (up == rt || upr == o || (up == o && upr == rt)));
        const bool ev = valid && o != dn && rt != dn && !(lane > 0 && (lf == dn || (lf == o && dlf == dn)));
        const bool ep = valid && o != rt && o != dn && o != dg && rt != dn && rt != dg && dn != dg;
        const unsigned mh = __ballot_sync(0xffffffffu, eh);
        const unsigned mv = __ballot_sync(0xffffffffu, ev);
        const unsigned mp = __ballot_sync(0xffffffffu, ep);
        if (mh | mv | mp) {
            // append this row's keys: horizontal, vertical, then plaquettes
            const int nh = __popc(mh), nv = __popc(mv);
            if (eh) link_list_put(list, n + __popc(mh & lt), edge_key(o, rt), P, D, inst);
            if (ev) link_list_put(list, n + nh + __popc(mv & lt), edge_key(o, dn), P, D, inst);
            if (ep) link_list_put(list, n + nh + nv + __popc(mp & lt), plaquette_key(o, rt, dg, dn, cq, MX, MY), P, D,
                                  inst);
            n += nh + nv + __popc(mp);
        }
        up = o;
        upr = rt;
        o = dn;
        rt = dg;
        lf = dlf;
    }
    __syncwarp();
    // equal keys within a round of 32 are merged; the tile's keys are
    // appended to the instance's link list (the link hash removes the rest)
    n = min(n, LSET);
    for (int kb = 0; kb < n; kb += 32) {
        const bool in = kb + lane < n;
        const unsigned long long key = in ? list[kb + lane] : EMPTY_KEY;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const bool has = in && lane == __ffs(grp) - 1;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        if (!m) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(&P.st[inst].n_eapp, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (has) {
            const int pos = base + __popc(m & lt);
            if (pos < D.edge_cap) P.ekeys[D.edge_off + pos] = key;
            else edge_global_insert(P, D, inst, key);   // list full: insert directly
        }
    }
}

// appended links -> link hash (+ degrees); appended pairs -> overlap hash

__global__ void k_merge_lists(Pools P, StepTable T) {
    const long long* pe = pre_arr(T, PRE_EA);
    const long long* po = pre_arr(T, PRE_OA);
    const long long ne = pe[T.n_act], no = po[T.n_act];
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ne + no;
         g += (long long)gridDim.x * blockDim.x) {
        if (g < ne) {
            const int a = seg_of(pe, T.n_act, g);
            const int inst = T.act[a];
            const InstDesc& D = P.desc[inst];
            edge_global_insert(P, D, inst, P.ekeys[D.edge_off + (g - pe[a])]);
        } else {
            const long long h = g - ne;
            const int a = seg_of(po, T.n_act, h);
            const int inst = T.act[a];
            const InstDesc& D = P.desc[inst];
            const long long j = D.ovl_off + (h - po[a]);
            ovl_global_insert(P, D, inst, P.oapp_key[j], P.oapp_cnt[j]);
        }
    }
}

void launch_merge_lists(const Launch& L) {
    launch_plan(L, 0);
    k_merge_lists<<<L.grid_items, 256, 0, L.s>>>(L.P, L.T);
    ++*L.nlaunch;
}

void launch_voronoi(const Launch& L) {
    k_voronoi<<<L.total_tilesV, VTHREADS, 0, L.s>>>(L.P, L.T);
    ++*L.nlaunch;
}

void launch_links(const Launch& L) {
    k_links<<<(L.total_tilesV + LINK_WARPS - 1) / LINK_WARPS, 32 * LINK_WARPS, 0, L.s>>>(L.P, L.T);
    ++*L.nlaunch;
}

}  // namespace vd
