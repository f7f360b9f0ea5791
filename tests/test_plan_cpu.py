"""CPU checks of the fused launch planner through ``sf_plan_launch`` (host
logic only, no device): every chosen shape fits in the opt-in shared memory
of a GB300 block, respects the launch bounds of the kernels and the
tensor-memory form's constraints (16-bit precisions: warps in groups of
four, the CTA's (sample, robot) rows within the 128 TMEM lanes, one partial
of F^T q per warp group, a sub-chunk's states within the 512 TMEM columns)
and takes no more samples per CTA than a scene has, and the bench workload
gets the shape measured fastest there."""
import math

import numpy as np
import pytest

SMEM_OPTIN = 232448   # bytes of opt-in shared memory per block on GB300
NUM_SMS = 152


@pytest.fixture(scope="module")
def plan():
    import paper_2501_19042_gb300 as P
    P.build()
    from paper_2501_19042_gb300.safety_filter import plan_launch
    return plan_launch


def test_bench_workload_shape(plan):
    """3D, N=16, S=1024, T=100: G=7 samples per CTA (147 CTAs, one wave on
    152 SMs), 11 warps, chunks of 50 steps, 3 time ranges: the shape a sweep
    on a GB300 measured fastest for the float32 form."""
    p = plan(3, 100, [16], [1024])
    assert (p["G"], p["warps"], p["tc"], p["nq"]) == (7, 11, 50, 3)
    assert p["smem"] <= SMEM_OPTIN
    assert math.ceil(1024 / p["G"]) <= NUM_SMS
    # 16-bit (tensor-memory) forms: G=7, 12 warps in 3 groups, chunks of 50
    for prec in ("bf16", "fp16"):
        q = plan(3, 100, [16], [1024], precision=prec)
        assert (q["G"], q["warps"], q["tc"], q["nq"]) == (7, 12, 50, 3)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_shapes_are_valid_for_random_scene_mixes(plan, prec):
    rng = np.random.default_rng(7)
    for _ in range(60):
        dim = int(rng.integers(2, 4))
        T = int(rng.choice([20, 37, 64, 100, 120, 200]))
        bucket = int(rng.choice([8, 16, 24, 32]))
        lo = {8: 1, 16: 9, 24: 17, 32: 25}[bucket]
        n_sc = int(rng.integers(1, 6))
        nr = [int(rng.integers(lo, bucket + 1)) for _ in range(n_sc)]
        ns = [int(rng.integers(1, 600)) for _ in range(n_sc)]
        p = plan(dim, T, nr, ns, precision=prec)
        assert 1 <= p["G"] <= 64
        assert 4 <= p["warps"] <= 12
        assert 1 <= p["tc"] <= T
        assert 1 <= p["nq"] <= p["tc"]
        assert 0 < p["smem"] <= SMEM_OPTIN
        if prec != "fp32":
            assert p["warps"] % 4 == 0 and p["nq"] == p["warps"] // 4
            assert p["G"] * bucket <= 128
            nsub = (p["tc"] + 63) // 64          # TMEM sub-chunks of <= 64 steps
            ts = (p["tc"] + nsub - 1) // nsub
            tcw = (ts + 15) // 16 * 16
            ka = 8   # 16-bit operands: 8 columns per 16 coefficients
            assert 2 * dim * tcw + 2 * dim * ka <= 512
            assert p["smem"] + 256 <= SMEM_OPTIN
        # G never exceeds the largest scene (a CTA holds samples of one scene)
        assert p["G"] <= max(ns)


def test_more_shared_memory_never_makes_a_shape_impossible(plan):
    for cap in (64 * 1024, 96 * 1024, 160 * 1024, SMEM_OPTIN):
        p = plan(3, 100, [16], [1024], smem_per_block_optin=cap)
        assert p["smem"] <= cap


def test_rejections(plan):
    from paper_2501_19042_gb300._native import SfError
    bad = [
        dict(dim=4, T=100, n_robots=[16], n_samples=[8]),       # dim
        dict(dim=3, T=1, n_robots=[16], n_samples=[8]),         # T
        dict(dim=3, T=100, n_robots=[33], n_samples=[8]),       # N > 32
        dict(dim=3, T=100, n_robots=[16, 20], n_samples=[8, 8]),  # two buckets in one group
        dict(dim=3, T=100, n_robots=[16], n_samples=[0]),       # no samples
        dict(dim=3, T=100, n_robots=[], n_samples=[]),          # no scenes
    ]
    for kw in bad:
        with pytest.raises(SfError) as e:
            plan(**kw)
        assert e.value.code == 1, kw
    with pytest.raises(SfError) as e:
        plan(3, 100, [32], [64], smem_per_block_optin=8 * 1024)   # nothing fits
    assert e.value.code == 6
