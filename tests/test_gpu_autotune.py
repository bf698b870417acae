"""The autotuner (EC_OPT_AUTOTUNE) times candidate plans on the first request
of a shape class, keeps the fastest per class, persists it as JSON when
EC_AUTOTUNE_CACHE is set, and never changes the curves."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_persists_a_plan(libec, tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path / "plans.json"
    monkeypatch.setenv("EC_AUTOTUNE_CACHE", str(cache))
    f, thr = workloads.config3(n=96, nblobs=30, L=257)
    want = oracle.ec_curves(f.numpy(), thr.numpy(), 257, 26, 13)
    ctx = ec.Context(0)
    ctx.set_option(ec.EC_OPT_AUTOTUNE, 1)
    fd, td = f.cuda(), thr.cuda()
    for _ in range(2):
        got = ec.curve(fd, td, descriptors=13, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want)
    plan = ctx.tuned_plan(3, ec.EC_F32, 257, 13, tuple(f.shape))
    assert plan is not None and plan[0] in (16, 32, 64)
    data = json.loads(cache.read_text())
    assert len(data) == 1 and list(data.values())[0][:3] == list(plan)
    ctx.close()
    # a new context finds the plan in the file without tuning
    ctx2 = ec.Context(0)
    assert ctx2.tuned_plan(3, ec.EC_F32, 257, 13, tuple(f.shape)) == plan
    g = workloads.quantize_u8(workloads.grf_2d(9, 300, 200, 3.0))
    ctx2.set_option(ec.EC_OPT_AUTOTUNE, 1)
    got2 = ec.curve(g.cuda(), None, L=256, descriptors=7, ctx=ctx2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got2.cpu().numpy(), oracle.ec_curves(g.numpy(), None, 256, 8, 7))
    assert len(json.loads(cache.read_text())) == 2
