"""The whole clustering of one fixed input captured as a CUDA graph
(abx_graph_*): every replay must give the oracle's labels for the current
contents of the point buffer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from cases import _clumpy  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2409_10743_gb300 import binding
    binding.lib()
    return binding


def _same(got, want, what):
    assert np.array_equal(got, want), f"{what}: {int((got != want).sum())} labels differ"


@pytest.mark.parametrize("minpts,eps,kw", [(2, 0.004, {}), (5, 0.006, dict(leaf_size=8, dense_cells=-1)),
                                           (2, 0.004, dict(dense_cells=1, leaf_size=2))])
def test_graph_replays_follow_the_buffer(abx, minpts, eps, kw):
    rng = np.random.default_rng(31 + minpts)
    p = _clumpy(rng, 60_000, 30, 0.01)
    t = torch.from_numpy(p).cuda()
    g = abx.Graph(t, eps, minpts, params=abx.Params(**kw) if kw else None)
    try:
        _same(g.launch().cpu().numpy(), oracle.dbscan(p, eps, minpts), "first replay")
        n0 = abx.launch_count()
        for k in range(2):  # new contents in the same buffer, replayed
            p2 = _clumpy(rng, 60_000, 30 + 10 * k, 0.01)
            t.copy_(torch.from_numpy(p2))
            lab = g.launch().cpu().numpy()
            _same(lab, oracle.dbscan(p2, eps, minpts), f"replay {k + 2}")
        assert abx.launch_count() - n0 >= 2 * 15  # each replay counts its kernels
        torch.cuda.synchronize()
        assert abx.device_status() == 0
        # the graph and a direct call agree on the same input
        direct = abx.dbscan(t, eps, minpts, params=abx.Params(**kw) if kw else None).cpu().numpy()
        _same(g.launch().cpu().numpy(), direct, "graph vs direct call")
    finally:
        g.close()


def test_graph_created_while_profiling(abx):
    """Profile events are not captured into the graph (profiling stays a
    property of direct calls)."""
    rng = np.random.default_rng(7)
    p = _clumpy(rng, 20_000, 10, 0.01)
    t = torch.from_numpy(p).cuda()
    abx.profile_enable(True)
    try:
        g = abx.Graph(t, 0.004, 2)
        lab = g.launch().cpu().numpy()
        g.close()
    finally:
        abx.profile_enable(False)
    _same(lab, oracle.dbscan(p, 0.004, 2), "graph under profiling")
