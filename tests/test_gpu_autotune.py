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


def _mixed_batch():
    reqs = workloads.request_stream(seed=11, n=24, max_2d=600, max_3d=80)
    fields = []
    for r in reqs:
        f, thr = workloads.request_field(r)
        fields.append(dict(field=f, thresholds=thr, L=r["L"], descriptors=7 if r["ndim"] == 2 else 15))
    return fields


def test_autotuned_batch_equals_oracle_and_keeps_a_plan(libec, tmp_path, monkeypatch):
    """The first batch of a mix class tunes (3D item depth, 2D item rows,
    grid) on itself; the tuned plan is kept per class, persisted, used by the
    next batch, and every run gives the oracle's curves."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path / "plans.json"
    monkeypatch.setenv("EC_AUTOTUNE_CACHE", str(cache))
    host = _mixed_batch()
    want = [oracle.ec_curves(d["field"].numpy(), None if d["thresholds"] is None else d["thresholds"].numpy(),
                             d["L"], 8 if d["field"].dim() == 2 else 26, d["descriptors"]) for d in host]
    dev = [dict(d, field=d["field"].cuda(), thresholds=None if d["thresholds"] is None else d["thresholds"].cuda())
           for d in host]
    ctx = ec.Context(0)
    ctx.set_option(ec.EC_OPT_AUTOTUNE, 1)
    b = ec.Batch(dev, ctx=ctx)
    assert b.tuned_plan() is None
    for _ in range(2):
        outs = b.run()
        torch.cuda.synchronize()
        for o, w in zip(outs, want):
            np.testing.assert_array_equal(o.cpu().numpy(), w)
    plan = b.tuned_plan()
    assert plan is not None
    tz3, grid, rows2d = plan
    assert tz3 in (16, 32, 64) and rows2d in (32, 64, 128) and grid >= 0
    data = json.loads(cache.read_text())
    keys = [k for k in data if k.startswith("batch_")]
    assert len(keys) == 1 and data[keys[0]][:3] == [tz3, grid, rows2d]
    # a server created on the tuning context shares its plans and gives the same curves
    sv = ec.Server(device_mem_budget=1 << 30, max_slots=2, ctx=ctx)
    tickets = sv.submit_many([dict(field=d["field"], thresholds=d["thresholds"], L=d["L"],
                                   descriptors=d["descriptors"]) for d in dev])
    for t, w in zip(tickets, want):
        np.testing.assert_array_equal(sv.wait(t), w)
    sv.close()
    ctx.close()


@pytest.mark.parametrize("tz3,rows2d,grid", [(16, 32, 0), (32, 128, 152), (64, 64, 1)])
def test_every_batch_plan_gives_the_same_curves(libec, tz3, rows2d, grid, tmp_path, monkeypatch):
    """Each candidate plan, forced through a pre-seeded tuning cache, gives
    the oracle's curves (plans change only speed)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    host = _mixed_batch()
    dev = [dict(d, field=d["field"].cuda(), thresholds=None if d["thresholds"] is None else d["thresholds"].cuda())
           for d in host]
    # learn the class key from a tuned run, then force the plan in the file
    cache = tmp_path / "plans.json"
    monkeypatch.setenv("EC_AUTOTUNE_CACHE", str(cache))
    scratch = ec.Context(0)
    scratch.set_option(ec.EC_OPT_AUTOTUNE, 1)
    ec.Batch(dev, ctx=scratch).run()
    torch.cuda.synchronize()
    scratch.close()
    data = json.loads(cache.read_text())
    key = [k for k in data if k.startswith("batch_")][0]
    data[key] = [tz3, grid, rows2d, 1.0]
    cache.write_text(json.dumps(data))
    ctx = ec.Context(0)
    ctx.set_option(ec.EC_OPT_AUTOTUNE, 1)
    b = ec.Batch(dev, ctx=ctx)
    assert b.tuned_plan() == (tz3, grid, rows2d)
    outs = b.run()
    torch.cuda.synchronize()
    for d, o in zip(host, outs):
        w = oracle.ec_curves(d["field"].numpy(), None if d["thresholds"] is None else d["thresholds"].numpy(),
                             d["L"], 8 if d["field"].dim() == 2 else 26, d["descriptors"])
        np.testing.assert_array_equal(o.cpu().numpy(), w)
    ctx.close()
