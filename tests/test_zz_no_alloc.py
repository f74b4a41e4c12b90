"""The allocation-free Voronoi entry point (vd_voronoi_owners_static).

It serves callers that cannot call cudaMalloc. Its owners must equal, site for
site, the owners the regular pipeline (vd_push_frame / vd_get_owners) computes
for the same centroids, on two calls in a row (the static scratch keeps the
previous call's contents, so the second call checks that it is cleared).
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1607_00908_gb300 import inputs as I  # noqa: E402
from paper_1607_00908_gb300 import vd  # noqa: E402


def _static_owners(cq: np.ndarray, Lx: int, Ly: int) -> np.ndarray:
    stream = torch.cuda.current_stream()
    d_cq = torch.from_numpy(np.ascontiguousarray(cq, dtype=np.int32)).cuda()
    d_out = torch.full((Ly, Lx), -7, dtype=torch.int32, device="cuda")
    st = vd.vd_voronoi_owners_static(d_cq.data_ptr() if cq.size else 0, int(cq.shape[0]), Lx, Ly,
                                     d_out.data_ptr(), stream.cuda_stream)
    assert st == vd.VD_OK, vd.status_string(st)
    stream.synchronize()
    return d_out.cpu().numpy()


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


def test_static_owners_rejects_too_many_centroids():
    cq = np.zeros((65537, 2), dtype=np.int32)
    d_out = torch.empty((8, 8), dtype=torch.int32, device="cuda")
    d_cq = torch.from_numpy(cq).cuda()
    st = vd.vd_voronoi_owners_static(d_cq.data_ptr(), 65537, 8, 8, d_out.data_ptr(), 0)
    assert st == vd.VD_ERR_CAPACITY
    assert vd.vd_voronoi_owners_static(d_cq.data_ptr(), 4, 0, 8, d_out.data_ptr(), 0) == vd.VD_ERR_INVALID
