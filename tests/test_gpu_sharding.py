"""The data-parallel split of a batch over ranks, run on one GPU: each
rank's shard (sharding.shard_batch: contiguous sample ranges, a scene cut by
a range boundary on both sides with its own start / goal rows) projected
serially gives, sample for sample, the same bits as the unsharded call.
Samples are independent problems (every reduction is per sample and the
exact pair pruning does not change any result), so the split needs no
collective on the data path."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_3D
from paper_2501_19042_gb300.sharding import shard_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("tm", [False, True])
def test_shards_equal_unsharded(sfmod, world, tm):
    """Scenes of one robot-count bucket (9..16 robots) and one forced launch
    shape for every call: the order of every reduction is then a function of
    the shape alone, so the bits cannot depend on which scenes share a
    launch."""
    P = sfmod
    scenes = si.ragged_batch(17, n_scenes=6, n_lo=9, n_hi=16, s_lo=5, s_hi=40, K=30)
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    xb = torch.tensor(np.concatenate([s.xi_bar.reshape(-1) for s in scenes]), dtype=torch.float32)
    st = torch.tensor(np.concatenate([s.start for s in scenes]), dtype=torch.float32)
    gl = torch.tensor(np.concatenate([s.goal for s in scenes]), dtype=torch.float32)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=16)
    f.set_tensor_memory(tm)
    f.set_launch_shape(4, 8 if tm else 11, 50)
    full = f.project(xb.cuda(), st.cuda(), gl.cuda(), 30, n_robots=nr, n_samples=ns)
    torch.cuda.synchronize()
    xi_full = full.xi.cpu()
    lam_full = full.lam.cpu()
    res_full = full.residual.cpu()
    coef_off = np.cumsum([0] + [3 * n * 11 * s for n, s in zip(nr, ns)])
    cut = 0
    for rank in range(world):
        sh = shard_batch(xb, st, gl, nr, ns, 3, rank, world)
        out = f.project(sh.xi_bar.cuda(), sh.start.cuda(), sh.goal.cuda(), 30, n_robots=sh.n_robots,
                        n_samples=sh.n_samples)
        torch.cuda.synchronize()
        xi, lam, res = out.xi.cpu(), out.lam.cpu(), out.residual.cpu()
        c = 0
        for (q, lo, hi), g0, N in zip(sh.scenes, sh.sample_offset, sh.n_robots):
            per = 3 * N * 11
            a, b = coef_off[q] + lo * per, coef_off[q] + hi * per
            assert torch.equal(xi[c: c + (hi - lo) * per], xi_full[a:b]), (rank, q)
            assert torch.equal(lam[c: c + (hi - lo) * per], lam_full[a:b]), (rank, q)
            c += (hi - lo) * per
            cut += int(lo > 0 or hi < ns[q])
        s0 = 0
        for (q, lo, hi), g0 in zip(sh.scenes, sh.sample_offset):
            assert torch.equal(res[s0: s0 + hi - lo], res_full[g0: g0 + hi - lo]), (rank, q)
            s0 += hi - lo
    assert cut > 0   # some scene is split between ranks
    f.sync_status()
