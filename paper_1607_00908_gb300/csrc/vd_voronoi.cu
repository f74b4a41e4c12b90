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
// Links: owners are computed for the tile plus one halo column and row, and
// a link {a, b} is emitted where a site and its +x or +y neighbour differ, and
// for a 2x2 plaquette with four distinct owners the diagonal chosen by the
// exact incircle test (int128). Links are deduplicated in a shared-memory set,
// then inserted into a global hash that also counts each label's degree.
#include "vd_internal.cuh"

namespace vd {

__device__ __forceinline__ long long floordiv_i(long long a, long long b) {
    long long d = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --d;
    return d;
}

// unwrapped bucket geometry along one axis (L sites, bucket side B, nb buckets)
__device__ __forceinline__ long long bucket_start(long long j, int L, int B, int nb) {
    const long long per = floordiv_i(j, nb);
    const long long jm = j - per * nb;
    return per * L + jm * B;
}
__device__ __forceinline__ long long bucket_end(long long j, int L, int B, int nb) {
    const long long per = floordiv_i(j, nb);
    const long long jm = j - per * nb;
    const long long e = (jm + 1) * B;
    return per * L + (e < L ? e : L);
}
__device__ __forceinline__ long long bucket_of_pos(long long p, int L, int B, int nb) {
    const long long per = floordiv_i(p, L);
    const long long pm = p - per * L;
    return per * nb + pm / B;
}

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
    unsigned h = (unsigned)hash64(key) & (unsigned)D.ehash_mask;
    for (int probe = 0; probe <= D.ehash_mask; ++probe) {
        const unsigned long long k = atomicCAS(&H[h], EMPTY_KEY, key);
        if (k == EMPTY_KEY) {
            const int idx = atomicAdd(&P.st[inst].n_edge_list, 1);
            if (idx < D.edge_cap) P.elist[D.edge_off + idx] = (int)h;
            else atomicOr(&P.st[inst].err, ERR_EDGE_CAP);
            atomicAdd(&P.deg[D.comp_off + (int)(key >> 32)], 1);
            return;
        }
        if (k == key) return;
        h = (h + 1) & (unsigned)D.ehash_mask;
    }
    atomicOr(&P.st[inst].err, ERR_EDGE_CAP);
}

__device__ __forceinline__ void edge_add(unsigned long long* s_set, const Pools& P, const InstDesc& D, int inst,
                                         unsigned long long key) {
    unsigned h = (unsigned)hash64(key) & (VEDGESET - 1);
    for (int probe = 0; probe < VEDGESET; ++probe) {
        const unsigned long long k = atomicCAS(&s_set[h], EMPTY_KEY, key);
        if (k == EMPTY_KEY || k == key) return;
        h = (h + 1) & (VEDGESET - 1);
    }
    edge_global_insert(P, D, inst, key);
}

__global__ __launch_bounds__(VTHREADS) void k_voronoi(Pools P, StepTable T) {
    __shared__ int s_cx[VCAND], s_cy[VCAND], s_id[VCAND];
    __shared__ long long s_md[VCAND];
    __shared__ int s_own[VH + 1][VW + 1];
    __shared__ unsigned long long s_set[VEDGESET];
    __shared__ int s_n;
    __shared__ int s_overflow;
    __shared__ long long s_U;

    const int b = blockIdx.x;
    const int a = seg_of_int(T.tileV_pre, T.n_act, b);
    const int inst = T.act[a];
    const InstDesc D = P.desc[inst];
    const InstState& S = P.st[inst];
    const int t = b - T.tileV_pre[a];
    const int tx = t % D.vtx, ty = t / D.vtx;
    const int x0 = tx * VW, y0 = ty * VH;
    const int ncols = min(VW, D.Lx - x0), nrows = min(VH, D.Ly - y0);
    const int now = S.slot ^ 1;
    const int K = min(S.K, D.comp_cap);
    const long long MX = (long long)Q * D.Lx, MY = (long long)Q * D.Ly;
    const int2* cq = P.cq + D.comp_off;

    for (int k = threadIdx.x; k < VEDGESET; k += VTHREADS) s_set[k] = EMPTY_KEY;
    if (threadIdx.x == 0) { s_n = 0; s_overflow = 0; }
    __syncthreads();

    if (K > 0 && threadIdx.x < 32) {
        // ---- candidate search (one warp) ----
        const int lane = threadIdx.x;
        const int Bk = S.B, nbx = S.nbx, nby = S.nby;
        const long long X0 = (long long)Q * x0, Y0 = (long long)Q * y0;
        const long long WR = (long long)Q * ncols, HR = (long long)Q * nrows;   // region incl. halo
        const long long bx0 = bucket_of_pos(x0, D.Lx, Bk, nbx), bx1 = bucket_of_pos(x0 + ncols, D.Lx, Bk, nbx);
        const long long by0 = bucket_of_pos(y0, D.Ly, Bk, nby), by1 = bucket_of_pos(y0 + nrows, D.Ly, Bk, nby);
        const int* boff = P.boff + D.bucket_off;
        const int2* bcq = P.bcq + D.comp_off;
        const int* bid = P.bid + D.comp_off;
        long long U = LLONG_MAX;
        long long px0 = 0, px1 = -1, py0 = 0, py1 = -1;
        bool pfx = false, pfy = false, have_prev = false;
        for (int r = 0;; ++r) {
            long long rx0 = bx0 - r, rx1 = bx1 + r, ry0 = by0 - r, ry1 = by1 + r;
            const bool fx = (rx1 - rx0 + 1) >= nbx, fy = (ry1 - ry0 + 1) >= nby;
            if (fx) { rx0 = 0; rx1 = nbx - 1; }
            if (fy) { ry0 = 0; ry1 = nby - 1; }
            const long long wx = rx1 - rx0 + 1, wy = ry1 - ry0 + 1;
            const long long ncell = wx * wy;
            for (long long k = lane; k < ncell; k += 32) {
                const long long cu = rx0 + k % wx, rv = ry0 + k / wx;
                if (have_prev) {
                    const bool inx = pfx || ((((cu - px0) % nbx) + nbx) % nbx) <= (px1 - px0);
                    const bool iny = pfy || ((((rv - py0) % nby) + nby) % nby) <= (py1 - py0);
                    if (inx && iny) continue;
                }
                const long long cm = ((cu % nbx) + nbx) % nbx, rm = ((rv % nby) + nby) % nby;
                const int bk = (int)(rm * nbx + cm);
                const int e = boff[bk + 1];
                for (int j = boff[bk]; j < e; ++j) {
                    const int2 c = bcq[j];
                    const long long ddx = wrapM((long long)c.x - X0, MX);
                    const long long ddy = wrapM((long long)c.y - Y0, MY);
                    const long long mnx = ring_mindist(ddx, WR, MX), mny = ring_mindist(ddy, HR, MY);
                    long long mxx = max(ddx < 0 ? -ddx : ddx, (ddx - WR) < 0 ? WR - ddx : ddx - WR);
                    long long mxy = max(ddy < 0 ? -ddy : ddy, (ddy - HR) < 0 ? HR - ddy : ddy - HR);
                    mxx = min(mxx, MX >> 1);
                    mxy = min(mxy, MY >> 1);
                    const long long mind = mnx * mnx + mny * mny;
                    const long long maxd = mxx * mxx + mxy * mxy;
                    if (maxd < U) U = maxd;
                    if (mind <= U) {
                        const int pos = atomicAdd(&s_n, 1);
                        if (pos < VCAND) {
                            s_cx[pos] = c.x;
                            s_cy[pos] = c.y;
                            s_id[pos] = bid[j];
                            s_md[pos] = mind;
                        } else {
                            s_overflow = 1;
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long v = __shfl_xor_sync(0xffffffffu, U, o);
                U = v < U ? v : U;
            }
            if (fx && fy) break;
            long long gx = LLONG_MAX, gy = LLONG_MAX;
            if (!fx) {
                const long long l = X0 - (long long)Q * bucket_start(rx0, D.Lx, Bk, nbx);
                const long long rr = (long long)Q * bucket_end(rx1, D.Lx, Bk, nbx) - (X0 + WR);
                gx = min(l, rr);
            }
            if (!fy) {
                const long long l = Y0 - (long long)Q * bucket_start(ry0, D.Ly, Bk, nby);
                const long long rr = (long long)Q * bucket_end(ry1, D.Ly, Bk, nby) - (Y0 + HR);
                gy = min(l, rr);
            }
            const long long g = min(gx, gy);
            // every unscanned centre is at least g away from the region
            if (g > 0 && g < (1ll << 31) && g * g > U) break;
            if (g >= (1ll << 31)) break;
            px0 = rx0; px1 = rx1; py0 = ry0; py1 = ry1; pfx = fx; pfy = fy; have_prev = true;
        }
        if (lane == 0) s_U = U;
    }
    __syncthreads();

    // ---- compact candidates to those within U ----
    const bool slow = (s_overflow != 0);
    int nc = min(s_n, VCAND);
    if (!slow && K > 0 && threadIdx.x < 32) {
        const long long U = s_U;
        int w = 0;
        for (int base = 0; base < nc; base += 32) {
            const int k = base + threadIdx.x;
            bool keep = false;
            int cx = 0, cy = 0, id = 0;
            long long md = 0;
            if (k < nc) {
                cx = s_cx[k]; cy = s_cy[k]; id = s_id[k]; md = s_md[k];
                keep = md <= U;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) {
                const int pos = w + __popc(m & ((1u << threadIdx.x) - 1u));
                s_cx[pos] = cx; s_cy[pos] = cy; s_id[pos] = id; s_md[pos] = md;
            }
            w += __popc(m);
            __syncwarp();
        }
        if (threadIdx.x == 0) s_n = w;
    }
    __syncthreads();
    nc = slow ? K : s_n;

    // ---- owners of the tile plus halo ----
    const int ew = ncols + 1, eh = nrows + 1;
    for (int k = threadIdx.x; k < ew * eh; k += VTHREADS) {
        const int lx = k % ew, ly = k / ew;
        const long long sx = (long long)Q * (x0 + lx), sy = (long long)Q * (y0 + ly);
        long long best = LLONG_MAX;
        int bi = -1;
        if (!slow) {
            for (int j = 0; j < nc; ++j) {
                const long long dx = wrapM(sx - s_cx[j], MX);
                const long long dy = wrapM(sy - s_cy[j], MY);
                const long long d2 = dx * dx + dy * dy;
                const int id = s_id[j];
                if (d2 < best || (d2 == best && id < bi)) { best = d2; bi = id; }
            }
        } else {
            for (int j = 0; j < K; ++j) {
                const int2 c = cq[j];
                const long long dx = wrapM(sx - c.x, MX);
                const long long dy = wrapM(sy - c.y, MY);
                const long long d2 = dx * dx + dy * dy;
                if (d2 < best) { best = d2; bi = j; }
            }
        }
        s_own[ly][lx] = bi;
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

    // ---- links ----
    if (K > 1) {
        for (int k = threadIdx.x; k < VW * VH / 4; k += VTHREADS) {
            const int ly = k / (VW / 4), lx0 = (k % (VW / 4)) * 4;
            if (ly >= nrows) continue;
            unsigned long long last = EMPTY_KEY;
            for (int i = 0; i < 4; ++i) {
                const int lx = lx0 + i;
                if (lx >= ncols) break;
                const int o = s_own[ly][lx], rt = s_own[ly][lx + 1];
                const int dn = s_own[ly + 1][lx], dg = s_own[ly + 1][lx + 1];
                if (o != rt) {
                    const unsigned long long kk = edge_key(o, rt);
                    if (kk != last) { edge_add(s_set, P, D, inst, kk); last = kk; }
                }
                if (o != dn) {
                    const unsigned long long kk = edge_key(o, dn);
                    if (kk != last) { edge_add(s_set, P, D, inst, kk); last = kk; }
                }
                if (o != rt && o != dn && o != dg && rt != dn && rt != dg && dn != dg) {
                    const unsigned long long kk = plaquette_key(o, rt, dg, dn, cq, MX, MY);
                    edge_add(s_set, P, D, inst, kk);
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < VEDGESET; k += VTHREADS)
            if (s_set[k] != EMPTY_KEY) edge_global_insert(P, D, inst, s_set[k]);
    }
    (void)now;
}

void launch_voronoi(const Launch& L) {
    k_voronoi<<<L.total_tilesV, VTHREADS, 0, L.s>>>(L.P, L.T);
    ++*L.nlaunch;
}

}  // namespace vd
