"""Seeded synthetic input fields for the detect pipeline.

The paper's production workload (Section 4) is the density field of a lattice
Boltzmann emulsion: about 2e3 droplets of diameter 30-35 sites on a 2048x1024
lattice. Those fields are not available, so the workloads here are synthetic
stand-ins of the same shape:

* ``smoothed_noise`` + ``shear_resample``: the "bubbles of a random field on a
  2D mesh" sample workload the paper mentions in Section 1. White noise is
  Gaussian-smoothed with periodic boundaries, normalised to unit standard
  deviation, and advanced frame to frame by a periodic affine shear plus small
  noise.
* ``rsa_discs`` + ``raster_discs``: an emulsion-like field of polydisperse
  discs (1.0 inside, 0.0 outside) placed by random sequential addition with a
  one-site minimum gap, advanced by an affine shear plus Gaussian jitter.

This module holds input generation only: it thresholds, labels and measures
nothing. Both the CUDA path and the CPU oracle consume the same float32 bytes
it produces. All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage

__all__ = [
    "smoothed_noise",
    "shear_resample",
    "noise_frames",
    "rsa_discs",
    "raster_discs",
    "disc_frames",
    "DiscState",
    "workload_c0",
    "workload_c1",
    "workload_c2",
    "batch_instances",
    "serve_sims",
]


def smoothed_noise(Ly: int, Lx: int, sigma: float, seed: int) -> np.ndarray:
    """White noise N(0,1), Gaussian-smoothed (periodic), scaled to unit std; float32."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((Ly, Lx))
    f = ndimage.gaussian_filter(w, sigma=sigma, mode="wrap")
    sd = f.std()
    if sd > 0:
        f = f / sd
    return f.astype(np.float32)


def shear_resample(F: np.ndarray, gamma: float, noise_std: float,
                   rng: np.random.Generator) -> np.ndarray:
    """Periodic bilinear backward resample under u_x = gamma*y, plus N(0, noise_std).

    Output(x, y) = F(x - gamma*y, y), x taken modulo Lx (the seam at y=0/Ly is
    kept, as a literal shear on the torus has one). Noise is added after the
    resample without renormalisation.
    """
    Ly, Lx = F.shape
    src = F.astype(np.float64)
    y = np.arange(Ly, dtype=np.float64)[:, None]
    x = np.arange(Lx, dtype=np.float64)[None, :]
    xs = x - gamma * y
    x0 = np.floor(xs)
    t = xs - x0
    i0 = np.mod(x0.astype(np.int64), Lx)
    i1 = np.mod(i0 + 1, Lx)
    rows = np.arange(Ly)[:, None]
    out = (1.0 - t) * src[rows, i0] + t * src[rows, i1]
    if noise_std > 0:
        out = out + noise_std * rng.standard_normal((Ly, Lx))
    return out.astype(np.float32)


def noise_frames(L: int, sigma: float, n_frames: int, gamma: float,
                 seed: int, noise_std: float = 0.01, Lx: int | None = None):
    """Yield ``n_frames`` float32 fields: a smoothed-noise frame, then sheared successors.

    Frame f+1 = shear_resample(frame f, gamma) + N(0, noise_std).
    """
    Ly = L
    Lx = L if Lx is None else Lx
    F = smoothed_noise(Ly, Lx, sigma, seed)
    rng = np.random.default_rng(seed + 7919)
    yield F
    for _ in range(n_frames - 1):
        F = shear_resample(F, gamma, noise_std, rng)
        yield F


# ----------------------------------------------------------------------------
# Emulsion-like disc fields
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class DiscState:
    L: int
    cx: np.ndarray   # float64 centres, [0, L)
    cy: np.ndarray
    r: np.ndarray    # radii
    attempts: int = 0

    @property
    def n(self) -> int:
        return int(self.cx.shape[0])

    @property
    def packing(self) -> float:
        return float(np.pi * np.sum(self.r ** 2) / (self.L * self.L))


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def rsa_discs(L: int, seed: int, rmin: float = 8.0, rmax: float = 12.0,
              gap: float = 1.0, max_consecutive_rejections: int = 200_000,
              batch: int = 8192, max_discs: int | None = None) -> DiscState:
    """Random sequential addition of discs on an L x L torus.

    A proposal (centre uniform in [0,L)^2, radius uniform in [rmin, rmax]) is
    accepted when every accepted disc satisfies |c - c'| >= r + r' + gap
    (minimum image). Proposals are drawn in batches from one seeded stream and
    judged strictly in order, so the result equals the one-at-a-time process.
    Stops after ``max_consecutive_rejections`` rejections in a row.
    """
    rng = np.random.default_rng(seed)
    cell = 2.0 * rmax + gap
    nc = max(1, int(L // cell))
    csz = L / nc
    per_cell = 8
    grid = -np.ones((nc, nc, per_cell), dtype=np.int64)
    fill = np.zeros((nc, nc), dtype=np.int64)
    cap = max(1024, int(2 * L * L / (np.pi * rmin * rmin)))
    cx = np.empty(cap)
    cy = np.empty(cap)
    rr = np.empty(cap)
    n = 0
    consecutive = 0
    attempts = 0
    offs = np.array([(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)])
    # Exact pre-filter: a unit cell is "blocked" when its centre lies closer
    # than rmin + r' + gap - sqrt(2)/2 to an accepted disc (c', r'); every
    # proposal whose centre falls in such a cell is certainly rejected.
    blocked = np.zeros((L, L), dtype=bool)
    W = int(math.ceil(rmin + rmax + gap)) + 1
    wo = np.arange(-W, W + 1)
    wox, woy = np.meshgrid(wo, wo)
    wox = wox.ravel()
    woy = woy.ravel()
    stamped = 0

    def stamp(upto):
        nonlocal stamped
        if upto <= stamped:
            return
        sx = np.floor(cx[stamped:upto]).astype(np.int64)
        sy = np.floor(cy[stamped:upto]).astype(np.int64)
        px_ = sx[:, None] + wox[None, :]
        py_ = sy[:, None] + woy[None, :]
        ddx = _min_image(px_ + 0.5 - cx[stamped:upto, None], L)
        ddy = _min_image(py_ + 0.5 - cy[stamped:upto, None], L)
        lim = rmin + rr[stamped:upto, None] + gap - math.sqrt(0.5) - 1e-9
        m = (lim > 0) & (ddx * ddx + ddy * ddy < lim * lim)
        blocked[np.mod(py_[m], L), np.mod(px_[m], L)] = True
        stamped = upto

    while consecutive < max_consecutive_rejections:
        if max_discs is not None and n >= max_discs:
            break
        stamp(n)
        px = rng.uniform(0.0, L, batch)
        py = rng.uniform(0.0, L, batch)
        pr = rng.uniform(rmin, rmax, batch)
        ok0 = ~blocked[np.minimum(py.astype(np.int64), L - 1), np.minimum(px.astype(np.int64), L - 1)]
        sv = np.flatnonzero(ok0)
        gx = np.minimum((px / csz).astype(np.int64), nc - 1)
        gy = np.minimum((py / csz).astype(np.int64), nc - 1)
        # survivors: exact check against the discs accepted before this batch
        ncx = (gx[sv, None] + offs[None, :, 0]) % nc
        ncy = (gy[sv, None] + offs[None, :, 1]) % nc
        cand = grid[ncy, ncx].reshape(sv.size, -1)
        valid = cand >= 0
        ci = np.where(valid, cand, 0)
        dx = _min_image(px[sv, None] - cx[ci], L)
        dy = _min_image(py[sv, None] - cy[ci], L)
        need = pr[sv, None] + rr[ci] + gap
        clash = valid & (dx * dx + dy * dy < need * need)
        ok0[sv[clash.any(axis=1)]] = False
        # Judge proposals in order. Those rejected by the pre-batch check only
        # extend the rejection run; survivors are re-checked against discs
        # accepted earlier in this batch.
        prev = -1
        stop = False
        for j in np.flatnonzero(ok0):
            run = j - prev - 1
            if consecutive + run >= max_consecutive_rejections:
                attempts += max_consecutive_rejections - consecutive
                consecutive = max_consecutive_rejections
                stop = True
                break
            consecutive += run
            attempts += run + 1
            prev = j
            accept = True
            for a, b in offs:
                cyi = (gy[j] + b) % nc
                cxi = (gx[j] + a) % nc
                for k in grid[cyi, cxi, :fill[cyi, cxi]]:
                    ddx = _min_image(px[j] - cx[k], L)
                    ddy = _min_image(py[j] - cy[k], L)
                    nd = pr[j] + rr[k] + gap
                    if ddx * ddx + ddy * ddy < nd * nd:
                        accept = False
                        break
                if not accept:
                    break
            if accept:
                if n >= cap or fill[gy[j], gx[j]] >= per_cell:
                    raise RuntimeError("RSA capacity exceeded")
                cx[n], cy[n], rr[n] = px[j], py[j], pr[j]
                grid[gy[j], gx[j], fill[gy[j], gx[j]]] = n
                fill[gy[j], gx[j]] += 1
                n += 1
                consecutive = 0
                if max_discs is not None and n >= max_discs:
                    stop = True
                    break
            else:
                consecutive += 1
                if consecutive >= max_consecutive_rejections:
                    stop = True
                    break
        if stop:
            break
        run = batch - prev - 1
        if consecutive + run >= max_consecutive_rejections:
            attempts += max_consecutive_rejections - consecutive
            consecutive = max_consecutive_rejections
            break
        consecutive += run
        attempts += run
    return DiscState(L=L, cx=cx[:n].copy(), cy=cy[:n].copy(), r=rr[:n].copy(),
                     attempts=attempts)


def raster_discs(state: DiscState) -> np.ndarray:
    """float32 field: 1.0 at sites whose min-image squared distance to a centre is < r^2."""
    L = state.L
    F = np.zeros((L, L), dtype=np.float32)
    if state.n == 0:
        return F
    R = int(math.ceil(float(state.r.max()))) + 1
    o = np.arange(-R, R + 1)
    ox, oy = np.meshgrid(o, o)
    ox = ox.ravel()
    oy = oy.ravel()
    step = 4096
    for s in range(0, state.n, step):
        cx = state.cx[s:s + step]
        cy = state.cy[s:s + step]
        r = state.r[s:s + step]
        bx = np.floor(cx).astype(np.int64)
        by = np.floor(cy).astype(np.int64)
        sx = bx[:, None] + ox[None, :]
        sy = by[:, None] + oy[None, :]
        dx = sx - cx[:, None]
        dy = sy - cy[:, None]
        inside = dx * dx + dy * dy < (r * r)[:, None]
        F[np.mod(sy[inside], L), np.mod(sx[inside], L)] = 1.0
    return F


def disc_frames(L: int, n_frames: int, seed: int, shear: float = 1e-3,
                jitter: float = 0.3, state: DiscState | None = None, **rsa_kw):
    """Yield (field, state) per frame: RSA discs, then c_x += shear*c_y and N(0, jitter) moves."""
    st = rsa_discs(L, seed, **rsa_kw) if state is None else state
    rng = np.random.default_rng(seed + 104729)
    cx, cy = st.cx.copy(), st.cy.copy()
    for f in range(n_frames):
        if f > 0:
            cx = cx + shear * cy + jitter * rng.standard_normal(cx.shape)
            cy = cy + jitter * rng.standard_normal(cy.shape)
            cx = np.mod(cx, L)
            cy = np.mod(cy, L)
        cur = DiscState(L=L, cx=cx, cy=cy, r=st.r, attempts=st.attempts)
        yield raster_discs(cur), cur


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def workload_c0(seed: int = 1):
    """128x128 smoothed noise, sigma 3, two frames; frame 2 = shear 0.02 + N(0, 0.01)."""
    return list(noise_frames(128, 3.0, 2, 0.02, seed))


def workload_c1(seed: int = 1, n_frames: int = 64):
    """1024x1024 smoothed noise, sigma 4; each frame a further shear 0.005 + N(0, 0.01)."""
    return noise_frames(1024, 4.0, n_frames, 0.005, seed)


def workload_c2(seed: int = 1, n_frames: int = 16, L: int = 4096, **rsa_kw):
    """4096x4096 RSA discs r~U[8,12], 1-site gap; shear 1e-3*y and N(0, 0.3) jitter per frame."""
    return disc_frames(L, n_frames, seed, **rsa_kw)


BATCH_SIZES = (256, 384, 512, 768, 1024, 1536, 2048)


def batch_instances(n: int = 256, seed: int = 3, sizes=BATCH_SIZES):
    """Instance parameters for the batched form: (L, sigma, seed_i) per instance."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(np.array(sizes), size=n)
    sig = rng.uniform(2.0, 6.0, size=n)
    return [(int(Ls[i]), float(sig[i]), int(seed * 100003 + i)) for i in range(n)]


def serve_sims(n: int = 64, seed: int = 5, sizes=(512, 1024, 2048, 4096)):
    """Simulation parameters for the served form: (L, recipe, seed_i); recipes alternate."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(np.array(sizes), size=n)
    return [(int(Ls[i]), "noise" if i % 2 == 0 else "discs", int(seed * 7919 + i))
            for i in range(n)]
