"""The allocation-free Voronoi entry point (vd_voronoi_owners_static).

It serves callers that cannot call cudaMalloc: processes whose device memory
all belongs to another framework's allocator, and real-time or embedded hosts
that allocate everything at start-up. Its scratch is one static device array
shared by every call, which keeps the previous call's contents.

Checked here: its owners equal, site for site, the owners the regular
pipeline (vd_push_frame / vd_get_owners) computes for the same centroids, on
two calls in a row; and they equal the oracle's brute-force argmin on cases
that reach every path of the kernel -- ragged lattices, windows that wrap
around a lattice with few centroids, a tile with more candidates than its
shared list holds (the scan over all centroids), no centroids, centroids
outside the lattice (ignored), a one-centroid-per-site strip at the maximum
count, and a lattice whose bucket grid must be widened to fit the scratch.
Consecutive cases of different sizes also check that each call clears what it
reuses. This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402

Q = 1024


def _static_owners(cq: np.ndarray, Lx: int, Ly: int) -> np.ndarray:
    stream = torch.cuda.current_stream()
    d_cq = torch.from_numpy(np.ascontiguousarray(cq, dtype=np.int32).reshape(-1, 2)).cuda()
    d_out = torch.full((Ly, Lx), -7, dtype=torch.int32, device="cuda")
    st = vd.vd_voronoi_owners_static(d_cq.data_ptr() if cq.size else 0, int(cq.shape[0]), Lx, Ly,
                                     d_out.data_ptr(), stream.cuda_stream)
    assert st == vd.VD_OK, vd.status_string(st)
    stream.synchronize()
    return d_out.cpu().numpy()


def _brute(cq: np.ndarray, Lx: int, Ly: int, sites=None) -> np.ndarray:
    """Oracle owners over the centroids inside [0, 1024 L), keeping their ids."""
    c = np.asarray(cq, dtype=np.int64).reshape(-1, 2)
    ok = (c[:, 0] >= 0) & (c[:, 1] >= 0) & (c[:, 0] < Q * Lx) & (c[:, 1] < Q * Ly)
    idx = np.flatnonzero(ok)
    o = O.owners_bruteforce(c[idx].astype(np.int32), Lx, Ly, sites=sites)
    return np.where(o >= 0, idx[np.maximum(o, 0)] if idx.size else -1, -1).astype(np.int32)


def _random_cq(rng, K, Lx, Ly):
    return np.stack([rng.integers(0, Q * Lx, K), rng.integers(0, Q * Ly, K)], axis=1).astype(np.int32)


def test_static_owners_equal_pipeline_owners_on_two_calls():
    assert torch.cuda.is_available()
    for Lx, Ly, frames in ((128, 128, I.workload_c0(seed=2)),
                           (200, 150, list(I.noise_frames(150, 3.0, 2, 0.02, seed=9, Lx=200)))):
        det = vd.Detector(Lx, Ly)
        for F in frames[:2]:
            det.push(torch.from_numpy(F).cuda())
            cq = det.centroids()
            want = det.owners()
            got = _static_owners(cq, Lx, Ly)
            assert np.array_equal(got, want)
        det.close()


def test_static_owners_equal_oracle_on_every_path():
    rng = np.random.default_rng(2024)
    # ragged lattice, against both tilings
    Lx, Ly = 203, 77
    cq = _random_cq(rng, 40, Lx, Ly)
    assert np.array_equal(_static_owners(cq, Lx, Ly), _brute(cq, Lx, Ly)), "ragged"
    # one to three centroids: every tile's window wraps around the lattice
    for K in (1, 2, 3):
        cq = _random_cq(rng, K, 150, 90)
        assert np.array_equal(_static_owners(cq, 150, 90), _brute(cq, 150, 90)), f"K={K}"
    # 1500 centroids packed in an 8 x 8-site patch plus 20 spread out: the
    # tiles around the patch collect more candidates than their shared list
    # holds and take the scan over all centroids
    L = 256
    packed = np.stack([rng.integers(Q * 100, Q * 108, 1500), rng.integers(Q * 100, Q * 108, 1500)], axis=1)
    cq = np.concatenate([_random_cq(rng, 20, L, L), packed]).astype(np.int32)
    assert np.array_equal(_static_owners(cq, L, L), _brute(cq, L, L)), "candidate overflow"
    # no centroids: every owner is -1 (after a call that wrote real owners)
    got = _static_owners(np.zeros((0, 2), np.int32), 64, 48)
    assert (got == -1).all(), "K=0"
    # centroids outside [0, 1024 L) are ignored; ids of the others are kept
    Lx, Ly = 128, 96
    cq = _random_cq(rng, 30, Lx, Ly)
    bad = np.array([[-1, 5], [5, -Q], [Q * Lx, 0], [0, Q * Ly], [Q * Lx + 77, Q * Ly + 3]], np.int32)
    cq = np.concatenate([cq[:10], bad, cq[10:]]).astype(np.int32)
    assert np.array_equal(_static_owners(cq, Lx, Ly), _brute(cq, Lx, Ly)), "outside centroids"


def test_static_owners_at_the_limits():
    rng = np.random.default_rng(7)
    # a 4096 x 16 strip with 65536 centroids (the maximum), some at equal
    # positions (ties to the smallest id); sampled sites against brute force
    Lx, Ly = 4096, 16
    cq = _random_cq(rng, 1 << 16, Lx, Ly)
    cq[1000:1010] = cq[5]
    got = _static_owners(cq, Lx, Ly).ravel()
    sites = rng.choice(Lx * Ly, size=2000, replace=False)
    assert np.array_equal(got[sites], _brute(cq, Lx, Ly, sites=sites)), "strip"
    # 1024 x 1100 with 65536 centroids: buckets of 4 sites would need 70400
    # cells, more than the scratch holds, so the bucket side is widened
    Lx, Ly = 1024, 1100
    cq = _random_cq(rng, 1 << 16, Lx, Ly)
    got = _static_owners(cq, Lx, Ly).ravel()
    sites = rng.choice(Lx * Ly, size=2000, replace=False)
    assert np.array_equal(got[sites], _brute(cq, Lx, Ly, sites=sites)), "widened grid"
    # the next, small call sees no trace of the large one
    cq = _random_cq(rng, 5, 40, 30)
    assert np.array_equal(_static_owners(cq, 40, 30), _brute(cq, 40, 30)), "small after large"


def test_static_owners_rejects_too_many_centroids():
    cq = np.zeros((65537, 2), dtype=np.int32)
    d_out = torch.empty((8, 8), dtype=torch.int32, device="cuda")
    d_cq = torch.from_numpy(cq).cuda()
    st = vd.vd_voronoi_owners_static(d_cq.data_ptr(), 65537, 8, 8, d_out.data_ptr(), 0)
    assert st == vd.VD_ERR_CAPACITY
    assert vd.vd_voronoi_owners_static(d_cq.data_ptr(), 4, 0, 8, d_out.data_ptr(), 0) == vd.VD_ERR_INVALID
