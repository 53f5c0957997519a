"""Launch shapes (ucp_launch_config) through the C ABI: every value of every
knob gives bit-identical controllers, winner positions, u1 tables and J, on
a batch of uneven instances and on one instance; the autotuner's choice is
one of them; out-of-range values are rejected."""
import numpy as np
import pytest

from paper_1908_04489_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CONFIGS = [
    {"search_lanes": 4}, {"search_lanes": 16},
    {"u1_threads": [1, 1, 1, 1, 1]}, {"u1_threads": [1, 2, 2, 2, 2]},
    {"u1_threads": [1, 2, 4, 4, 4]},
    {"defer_blocks": 1}, {"defer_blocks": 64},
    {"search_lanes": 16, "u1_threads": [1, 2, 2, 1, 2], "defer_blocks": 3},
]


@pytest.fixture(scope="module")
def binding():
    import torch
    assert torch.cuda.is_available()
    from paper_1908_04489_gb300 import binding as b, build
    build.build()
    b.load()
    return b


def mixed(n, seed=29):
    rng = W.SplitMix64(seed, 7)
    return [W.random_instance(rng, (0.1, 0.05), 3, 1) for _ in range(n)]


def batch_state(binding, ps, cfg, stream):
    with binding.Batch(ps, stream=stream) as b:
        if cfg is not None:
            b.set_launch_config(cfg)
        b.sweep(3)
        return [(m.get_controllers(), m.J_history()) for m in b.members]


def test_every_launch_shape_gives_the_same_batch(binding):
    import torch
    stream = torch.cuda.Stream()
    ps = mixed(6)
    ref = batch_state(binding, ps, None, stream)
    for cfg in CONFIGS:
        got = batch_state(binding, ps, cfg, stream)
        for (a, Ja), (b, Jb) in zip(got, ref):
            for k in ("f", "U", "idx"):
                np.testing.assert_array_equal(a[k], b[k], err_msg=str(cfg))
            np.testing.assert_array_equal(Ja, Jb, err_msg=str(cfg))


@pytest.mark.parametrize("use_stream", [True, False])
def test_every_launch_shape_gives_the_same_instance(binding, use_stream):
    import torch
    p = W.c1() | {"precision": 1}
    stream = torch.cuda.Stream() if use_stream else None

    def run(cfg):
        with binding.Instance(p, stream=stream) as inst:
            if cfg is not None:
                inst.set_launch_config(cfg)
            inst.sweep(3)
            return inst.get_controllers(), inst.J_history()

    ref, Jr = run(None)
    for cfg in CONFIGS:
        got, Jg = run(cfg)
        for k in ("f", "U", "idx"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=str(cfg))
        np.testing.assert_array_equal(Jg, Jr, err_msg=str(cfg))


def test_autotuner_picks_a_valid_shape_and_caches_it(binding, tmp_path):
    import torch
    from paper_1908_04489_gb300 import autotune as A
    stream = torch.cuda.Stream()
    ps = mixed(8, seed=31)
    path = str(tmp_path / "cache.json")
    cfg, table = A.tuned_batch_config(binding, ps, stream, "test-gpu", path=path,
                                      sweeps=1, reps=1)
    assert table and all(ms > 0 for _, ms in table)
    again, none = A.tuned_batch_config(binding, ps, stream, "test-gpu", path=path)
    assert again == cfg and none is None
    ref = batch_state(binding, ps, None, stream)
    got = batch_state(binding, ps, cfg, stream)
    for (a, Ja), (b, Jb) in zip(got, ref):
        np.testing.assert_array_equal(a["f"], b["f"])
        np.testing.assert_array_equal(Ja, Jb)


def test_out_of_range_shapes_are_rejected(binding):
    with binding.Instance(W.small()) as inst:
        for bad in ({"search_lanes": 5}, {"u1_threads": [2, 0, 0, 0, 0]},
                    {"u1_threads": [0, 0, 0, 0, 8]}, {"defer_blocks": -1},
                    {"defer_blocks": 5000}):
            with pytest.raises(binding.UcpError):
                inst.set_launch_config(bad)
        inst.sweep(1)
