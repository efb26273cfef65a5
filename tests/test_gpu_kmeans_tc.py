"""GPU checks of the tensor-core k-means assignment (Sec. III-A's assignment
step on tcgen05, csrc/kmeans_tc.cu), which a BF16 index uses:
  * after a fit, every user's centroid is a nearest fitted centroid within
    the BF16 bound of the objective u . c - ||c||^2 / 2 (checked against all
    fitted centroids, not only the kept ones), across several 256-centroid
    chunks with a ragged last chunk and operand rows of one and two
    64-element chunks;
  * Maximus stays equal to the oracle on those clusterings;
  * k-means itself on the tensor-core path: every final centroid is the mean
    of its members, and the FP32 index (CUDA-core assignment) agrees on most
    users."""
import numpy as np
import pytest

from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle
from test_gpu_fit import kmeans_err_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# (every case keeps its centroids resident: 256-centroid chunks x 64-element row chunks fit shared memory)
@pytest.mark.parametrize("f,C", [(24, 300), (100, 400), (51, 64), (7, 1)])
def test_fitted_assignment_is_near_optimal(f, C):
    U = synth.clustered_users(3000, f, 21, n_dirs=40, noise=0.3)
    I = synth.gaussian_rows(1200, f, 21, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.7))
    K = 10
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=C, dtype="bf16")
    mips.fit_clusters(index, torch.from_numpy(U).cuda())
    Cf = min(C, U.shape[0])
    fit = mips.get_buffer(index, "fit_centroids", torch.float32, (Cf, f)).cpu().numpy().astype(np.float64)
    idx, sc = mips.topk_maximus(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy())
    Ce = mips.get_stats(index)["clusters"]
    assign = mips.get_buffer(index, "assign", torch.int32, (U.shape[0],)).cpu().numpy()
    kept = mips.get_buffer(index, "centroids", torch.float32, (Ce, f)).cpu().numpy().astype(np.float64)
    # each kept slot is a copy of one fitted centroid: find it
    rows = {fit[j].tobytes(): j for j in range(Cf)}
    slot_to_fit = np.array([rows[kept[s].tobytes()] for s in range(Ce)])
    a = slot_to_fit[assign]
    U64 = U.astype(np.float64)
    obj = U64 @ fit.T - 0.5 * (fit * fit).sum(axis=1)[None, :]
    e = kmeans_err_bound(U64, fit)
    r = np.arange(U.shape[0])
    assert (obj[r, a] + e[r, a] >= (obj - e).max(axis=1)).all()
    index.close()


def test_kmeans_on_tensor_cores_matches_cuda_cores_mostly():
    U = synth.clustered_users(4000, 51, 5, n_dirs=32, noise=0.2)
    I = synth.gaussian_rows(2000, 51, 5, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.7))
    K, C = 10, 32
    out = {}
    for dtype in ("bf16", "fp32"):
        index = mips.build_index(torch.from_numpy(I).cuda(), clusters=C, dtype=dtype, kmeans_iters=1)
        idx, sc = mips.topk_maximus(index, torch.from_numpy(U).cuda(), K)
        mips.sync(index)
        check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy())
        Ce = mips.get_stats(index)["clusters"]
        a = mips.get_buffer(index, "assign", torch.int32, (U.shape[0],)).cpu().numpy()
        cent = mips.get_buffer(index, "centroids", torch.float32, (Ce, 51)).cpu().numpy().astype(np.float64)
        for j in range(Ce):  # the final centroids are their members' means
            m = a == j
            if m.any():
                np.testing.assert_allclose(cent[j], U.astype(np.float64)[m].mean(axis=0), rtol=1e-4, atol=1e-5)
        out[dtype] = a
        index.close()
    # one step from the same seeded initial centroids: the two assignments
    # differ only where two centroids are within the BF16 rounding
    assert (out["bf16"] == out["fp32"]).mean() > 0.9
