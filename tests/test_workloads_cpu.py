"""Host-side checks of the served workload's generators and of the bench's
stratified oracle subset (no GPU): the request stream has the stated mix and
sizes, the device generator's recipe gives fields of the right shape, type
and spread (run here on the CPU), and the subset covers every side quartile
of both kinds plus the largest field of each."""
import sys
from pathlib import Path

import numpy as np
import torch

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402
from paper_2311_11740_gb300 import workloads  # noqa: E402


def test_request_stream_mix_and_sizes():
    reqs = workloads.request_stream(seed=5, n=4096, max_2d=4096, max_3d=512)
    assert len(reqs) == 4096
    two = [r for r in reqs if r["ndim"] == 2]
    three = [r for r in reqs if r["ndim"] == 3]
    assert 0.67 < len(two) / len(reqs) < 0.73
    assert all(64 <= r["side"] <= 4096 and r["dtype"] == "u8" and r["L"] == 256 for r in two)
    assert all(32 <= r["side"] <= 512 and r["dtype"] == "f32" and 64 <= r["L"] <= 1024 for r in three)
    assert all(2 <= r["sigma"] <= 10 for r in reqs)
    t = [r["arrival_s"] for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    # log-uniform sides: about half of each kind below the geometric mean of its range
    assert 0.4 < np.mean([r["side"] < 512 for r in two]) < 0.6
    assert 0.4 < np.mean([r["side"] < 128 for r in three]) < 0.6


def test_device_generator_recipe_on_the_host():
    for req in (dict(ndim=2, side=77, sigma=3.0, L=256, seed=11), dict(ndim=3, side=33, sigma=2.5, L=100, seed=12),
                dict(ndim=2, side=64, sigma=9.0, L=256, seed=13)):
        f, thr = workloads.request_field_device(req, device="cpu")
        assert tuple(f.shape) == (req["side"],) * req["ndim"] and f.is_contiguous()
        if req["ndim"] == 2:
            assert f.dtype == torch.uint8 and thr is None
            assert int(f.min()) == 0 and int(f.max()) == 255   # quantised over [min, max]
        else:
            assert f.dtype == torch.float32 and thr.numel() == req["L"]
            t = thr.numpy()
            assert np.all(np.diff(t) > 0) and t[0] == f.min().item() and t[-1] == f.max().item()
        g, _ = workloads.request_field_device(req, device="cpu")
        assert torch.equal(f, g)   # seeded


def test_stratified_oracle_subset_covers_quartiles_and_extremes():
    reqs = workloads.request_stream(seed=5, n=4096, max_2d=4096, max_3d=512)
    sub = bench.stratified_subset(reqs, 32, 5)
    assert len(sub) >= 256 and len(set(sub)) == len(sub)
    for nd in (2, 3):
        idx = sorted((i for i, r in enumerate(reqs) if r["ndim"] == nd), key=lambda i: reqs[i]["side"])
        assert idx[-1] in sub   # the largest field of the kind
        for q in range(4):
            part = set(idx[len(idx) * q // 4:len(idx) * (q + 1) // 4])
            assert len(part & set(sub)) >= 32
