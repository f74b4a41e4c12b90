// Voronoi owners with no device allocation (vd_voronoi_owners_static).
//
// Some callers cannot call cudaMalloc: processes whose device memory is all
// handed out to another framework's allocator (a device allocation there
// fails, or takes memory that allocator counts on), and real-time or embedded
// hosts that allocate everything once at start-up and may not allocate (or
// risk the implicit synchronisation of an allocation) afterwards.
// This entry point computes the same exact digital Voronoi colouring as the
// detect pipeline (Section 3.2.1 of the paper: every site takes the label of
// the nearest centre by exact squared distance, minimum image on the torus,
// ties to the smallest label) from caller-provided centroids into a
// caller-provided owner array, using only the fixed scratch below.
//
// Scratch: one file-scope __device__ array, sizeof(NoAllocScratch) =
// 1,572,868 bytes (about 1.5 MB), present on every GPU that loads the library
// until the process exits. It holds the centroid bucket grid (counts, offsets, centroids in
// bucket order). Every call shares it and it keeps the last call's contents;
// the call clears what must start at zero. Calls whose device work overlaps
// (different streams, or several host threads) race on it: serialise them.
// The array's device address is resolved once per device, by the first call
// made with that device current; resetting the device (cudaDeviceReset)
// invalidates it, so the entry point must not be used across a reset.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "vd.h"

namespace {

constexpr int NA_MAX_K = 1 << 16;          // centroids per call
constexpr int NA_MAX_BUCKETS = 1 << 16;    // bucket grid cells
constexpr int NA_Q = 1024;
constexpr int NA_TW = 32, NA_TH = 32;
constexpr int NA_CAND = 1024;
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    int bcnt[NA_MAX_BUCKETS];
    int boff[NA_MAX_BUCKETS + 1];
    int cursor[NA_MAX_BUCKETS];
    int2 bcq[NA_MAX_K];
    int bid[NA_MAX_K];
};

__device__ __align__(256) NoAllocScratch g_na_scratch;

__device__ __forceinline__ long long na_wrap(long long d, long long M) {
    const long long h = M >> 1;
    if (d >= h) d -= M;
    else if (d < -h) d += M;
    return d;
}

__device__ __forceinline__ long long na_floordiv(long long a, long long b) {
    long long d = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --d;
    return d;
}
// unwrapped extent [start, end) of bucket column j (any integer) on a ring of L
// sites cut into nb buckets of side B, the last one possibly narrower
__device__ __forceinline__ long long na_bstart(long long j, int L, int B, int nb) {
    const long long per = na_floordiv(j, nb);
    return per * L + (j - per * nb) * B;
}
__device__ __forceinline__ long long na_bend(long long j, int L, int B, int nb) {
    const long long per = na_floordiv(j, nb);
    const long long e = (j - per * nb + 1) * B;
    return per * L + (e < L ? e : L);
}

__global__ void na_clear(NoAllocScratch* S, int nb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        S->bcnt[i] = 0;
        S->cursor[i] = 0;
    }
}

__device__ __forceinline__ bool na_inside(int2 c, int Lx, int Ly) {
    return c.x >= 0 && c.y >= 0 && c.x / NA_Q < Lx && c.y / NA_Q < Ly;
}

__global__ void na_count(NoAllocScratch* S, const int2* cq, int K, int B, int nbx, int Lx, int Ly) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
        const int2 c = cq[i];
        if (!na_inside(c, Lx, Ly)) continue;   // outside [0, 1024*L): ignored
        atomicAdd(&S->bcnt[((c.y / NA_Q) / B) * nbx + (c.x / NA_Q) / B], 1);
    }
}

// one block: exclusive scan of nb <= NA_MAX_BUCKETS counts
__global__ void na_scan(NoAllocScratch* S, int nb) {
    __shared__ int s_part[1024];
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += S->bcnt[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = s_part[t];
            s_part[t] = run;
            run += v;
        }
        S->boff[nb] = run;
    }
    __syncthreads();
    int run = s_part[threadIdx.x];
    for (int i = lo; i < hi; ++i) {
        S->boff[i] = run;
        run += S->bcnt[i];
    }
}

__global__ void na_scatter(NoAllocScratch* S, const int2* cq, int K, int B, int nbx, int Lx, int Ly) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
        const int2 c = cq[i];
        if (!na_inside(c, Lx, Ly)) continue;
        const int b = ((c.y / NA_Q) / B) * nbx + (c.x / NA_Q) / B;
        const int pos = S->boff[b] + atomicAdd(&S->cursor[b], 1);
        S->bcq[pos] = c;
        S->bid[pos] = i;
    }
}

// owners of one 32 x 32 tile: candidates from whole bucket rings until the
// unscanned region is farther than the best upper bound, then exact argmin
__global__ void na_owners(const NoAllocScratch* S, const int2* cq, int K, int Lx, int Ly, int B, int nbx,
                          int nby, int* owners) {
    __shared__ int s_cx[NA_CAND], s_cy[NA_CAND], s_id[NA_CAND];
    __shared__ int s_n, s_over;
    __shared__ unsigned long long s_U;
    const int vtx = (Lx + NA_TW - 1) / NA_TW;
    const int tx = blockIdx.x % vtx, ty = blockIdx.x / vtx;
    const int x0 = tx * NA_TW, y0 = ty * NA_TH;
    const int nc = min(NA_TW, Lx - x0), nr = min(NA_TH, Ly - y0);
    const long long MX = (long long)NA_Q * Lx, MY = (long long)NA_Q * Ly;
    const long long X0 = (long long)NA_Q * x0, Y0 = (long long)NA_Q * y0;
    const long long W = (long long)NA_Q * (nc - 1), H = (long long)NA_Q * (nr - 1);
    if (threadIdx.x == 0) {
        s_n = 0;
        s_over = 0;
        s_U = ULLONG_MAX;
    }
    __syncthreads();
    const int bx0 = x0 / B, bx1 = (x0 + nc - 1) / B, by0 = y0 / B, by1 = (y0 + nr - 1) / B;
    for (int r = 0;; ++r) {
        // whole rectangle of buckets within Chebyshev distance r (each bucket once)
        const int wx = min(nbx, bx1 - bx0 + 1 + 2 * r), wy = min(nby, by1 - by0 + 1 + 2 * r);
        const int rx0 = (wx == nbx) ? 0 : bx0 - r, ry0 = (wy == nby) ? 0 : by0 - r;
        const int pwx = (r == 0) ? 0 : min(nbx, bx1 - bx0 + 2 * r - 1), pwy = (r == 0) ? 0 : min(nby, by1 - by0 + 2 * r - 1);
        const int prx0 = (pwx == nbx) ? 0 : bx0 - (r - 1), pry0 = (pwy == nby) ? 0 : by0 - (r - 1);
        for (int k = threadIdx.x; k < wx * wy; k += blockDim.x) {
            const int cu = rx0 + k % wx, rv = ry0 + k / wx;
            if (r > 0) {
                const bool inx = ((cu - prx0) % nbx + nbx) % nbx < pwx;
                const bool iny = ((rv - pry0) % nby + nby) % nby < pwy;
                if (inx && iny) continue;
            }
            const int b = ((rv % nby + nby) % nby) * nbx + ((cu % nbx + nbx) % nbx);
            for (int j = S->boff[b]; j < S->boff[b + 1]; ++j) {
                const int2 c = S->bcq[j];
                const long long dx = na_wrap((long long)c.x - X0, MX), dy = na_wrap((long long)c.y - Y0, MY);
                const long long ax = max(dx < 0 ? -dx : dx, dx > W ? dx - W : W - dx);
                const long long ay = max(dy < 0 ? -dy : dy, dy > H ? dy - H : H - dy);
                const long long mx = min(ax, MX >> 1), my = min(ay, MY >> 1);
                atomicMin(&s_U, (unsigned long long)(mx * mx + my * my));
                const int pos = atomicAdd(&s_n, 1);
                if (pos < NA_CAND) {
                    s_cx[pos] = c.x;
                    s_cy[pos] = c.y;
                    s_id[pos] = S->bid[j];
                } else {
                    s_over = 1;
                }
            }
        }
        __syncthreads();
        if (wx == nbx && wy == nby) break;
        // distance from the tile to the nearest unscanned bucket (buckets are B wide, the last may be narrower)
        long long g = LLONG_MAX;
        if (wx < nbx)
            g = min(g, min(X0 - (long long)NA_Q * na_bstart(bx0 - r, Lx, B, nbx),
                           (long long)NA_Q * na_bend(bx1 + r, Lx, B, nbx) - (X0 + W)));
        if (wy < nby)
            g = min(g, min(Y0 - (long long)NA_Q * na_bstart(by0 - r, Ly, B, nby),
                           (long long)NA_Q * na_bend(by1 + r, Ly, B, nby) - (Y0 + H)));
        const unsigned long long U = s_U;
        __syncthreads();
        if (g > 0 && (unsigned long long)g * (unsigned long long)g > U) break;
    }
    const bool all = s_over != 0;
    const int n = all ? K : s_n;
    for (int k = threadIdx.x; k < nc * nr; k += blockDim.x) {
        const int lx = k % nc, ly = k / nc;
        const long long sx = (long long)NA_Q * (x0 + lx), sy = (long long)NA_Q * (y0 + ly);
        long long best = LLONG_MAX;
        int bi = -1;
        for (int j = 0; j < n; ++j) {
            if (all && !na_inside(cq[j], Lx, Ly)) continue;
            const int cx = all ? cq[j].x : s_cx[j], cy = all ? cq[j].y : s_cy[j], id = all ? j : s_id[j];
            const long long dx = na_wrap(sx - cx, MX), dy = na_wrap(sy - cy, MY);
            const long long d2 = dx * dx + dy * dy;
            if (d2 < best || (d2 == best && id < bi)) {
                best = d2;
                bi = id;
            }
        }
        owners[(long long)(y0 + ly) * Lx + x0 + lx] = bi;
    }
}

// launch with the launch's own error (a stale error left by unrelated work in
// the process is neither reported as this call's nor cleared)
template <typename... KArgs, typename... Args>
cudaError_t na_launch(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

std::mutex g_na_mu;
NoAllocScratch* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

}  // namespace

extern "C" vd_status vd_voronoi_owners_static(const int32_t* d_centroids_q10, int32_t K, int32_t Lx, int32_t Ly,
                                              int32_t* d_owners, void* stream) {
    if (Lx < 1 || Ly < 1 || Lx >= (1 << 21) || Ly >= (1 << 21) || (long long)Lx * Ly >= (1ll << 31))
        return VD_ERR_INVALID;
    if (K < 0 || !d_owners || (K > 0 && !d_centroids_q10)) return VD_ERR_INVALID;
    if (K > NA_MAX_K) return VD_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return VD_ERR_CUDA;
    NoAllocScratch* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            // first call on this device: resolve the scratch array's device address
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess) return VD_ERR_CUDA;
            g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
        }
        S = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = (long long)Lx * Ly;
    const int tiles = ((Lx + NA_TW - 1) / NA_TW) * ((Ly + NA_TH - 1) / NA_TH);
    if (K == 0) {
        if (cudaMemsetAsync(d_owners, 0xff, sizeof(int32_t) * N, s) != cudaSuccess) return VD_ERR_CUDA;
        return VD_OK;
    }
    // bucket side ~ centre spacing, at least 4 sites, small enough to fit the scratch grid
    int B = (int)(sqrt((double)N / (double)K) + 0.5);
    if (B < 4) B = 4;
    while ((long long)((Lx + B - 1) / B) * ((Ly + B - 1) / B) > NA_MAX_BUCKETS) ++B;
    const int nbx = (Lx + B - 1) / B, nby = (Ly + B - 1) / B, nb = nbx * nby;
    const int2* cq = reinterpret_cast<const int2*>(d_centroids_q10);
    // each launch is checked before the next one is enqueued
    if (na_launch(na_clear, 64, 256, s, S, nb) != cudaSuccess) return VD_ERR_CUDA;
    if (na_launch(na_count, 64, 256, s, S, cq, K, B, nbx, Lx, Ly) != cudaSuccess) return VD_ERR_CUDA;
    if (na_launch(na_scan, 1, 1024, s, S, nb) != cudaSuccess) return VD_ERR_CUDA;
    if (na_launch(na_scatter, 64, 256, s, S, cq, K, B, nbx, Lx, Ly) != cudaSuccess) return VD_ERR_CUDA;
    if (na_launch(na_owners, tiles, 256, s, (const NoAllocScratch*)S, cq, K, Lx, Ly, B, nbx, nby, d_owners) !=
        cudaSuccess)
        return VD_ERR_CUDA;
    return VD_OK;
}
