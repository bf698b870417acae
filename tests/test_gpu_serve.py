"""The request loop (ec_server_*): requests admitted while others run give
the same curves as standalone calls and as the oracle; admission respects the
device-memory budget and slots; host-side failures surface as statuses."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ec.Context(0)


def _requests(n, seed=5, max_2d=600, max_3d=72):
    reqs = workloads.request_stream(seed=seed, n=n, max_2d=max_2d, max_3d=max_3d)
    out = []
    for r in reqs:
        f, thr = workloads.request_field(r)
        desc = 7 if r["ndim"] == 2 else 15
        out.append((f.numpy(), None if thr is None else thr.numpy(), r["L"], desc))
    return out


def test_served_mix_equals_standalone_and_oracle(ctx):
    reqs = _requests(48)
    sv = ec.Server(device_mem_budget=256 << 20, max_slots=4, ctx=ctx)
    tickets = [sv.submit(f, thr, L=L, descriptors=d) for f, thr, L, d in reqs]
    for t, (f, thr, L, d) in zip(tickets, reqs):
        got = sv.wait(t, timeout_ms=120000)
        want = oracle.ec_curves(f, thr, L, 8 if f.ndim == 2 else 26, d)
        np.testing.assert_array_equal(got, want)
        alone = ec.curve(torch.from_numpy(f).cuda(), None if thr is None else torch.from_numpy(thr).cuda(),
                         L=L, descriptors=d, ctx=ctx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got, alone.cpu().numpy())
    st = sv.stats()
    assert st["count"] == len(reqs)
    assert 0 < st["p50_us"] <= st["p99_us"]
    sv.close()


def test_served_pinned_torch_fields(ctx):
    # page-locked torch fields with numpy thresholds, as a serving front end passes them
    reqs = _requests(12, seed=9)
    sv = ec.Server(device_mem_budget=256 << 20, max_slots=4, ctx=ctx)
    tickets = [sv.submit(torch.from_numpy(f).pin_memory(), thr, L=L, descriptors=d) for f, thr, L, d in reqs]
    for t, (f, thr, L, d) in zip(tickets, reqs):
        np.testing.assert_array_equal(sv.wait(t, timeout_ms=120000),
                                      oracle.ec_curves(f, thr, L, 8 if f.ndim == 2 else 26, d))
    sv.close()


def test_submit_many_is_all_or_none(ctx):
    reqs = _requests(20, seed=11)
    sv = ec.Server(device_mem_budget=256 << 20, max_slots=3, ctx=ctx)
    tickets = sv.submit_many(reqs)
    assert len(tickets) == len(reqs) and len(set(tickets)) == len(reqs)
    sv.wait_all(120000)
    for t, (f, thr, L, d) in zip(tickets, reqs):
        assert sv.poll(t) == (True, 0)
        np.testing.assert_array_equal(sv.result(t), oracle.ec_curves(f, thr, L, 8 if f.ndim == 2 else 26, d))
    # one malformed request rejects the whole burst, naming its index
    bad = list(reqs[:3]) + [dict(field=reqs[0][0], thresholds=reqs[0][1], L=reqs[0][2], descriptors=7,
                                 connectivity=5)]
    with pytest.raises(ec.ECError) as e:
        sv.submit_many(bad)
    assert e.value.status == 1 and "request 3" in str(e.value)
    assert sv.stats()["count"] == len(reqs)
    sv.close()


def test_admission_budget_slots_and_failures(ctx):
    big = workloads.config3(n=160, nblobs=50, L=300)
    f, thr = big[0].numpy(), big[1].numpy()
    need = f.nbytes + thr.nbytes + 4 * 300 * 8 * 2 + 4096
    sv = ec.Server(device_mem_budget=need + (1 << 20), max_slots=1, ctx=ctx)
    a = sv.submit(f, thr, descriptors=15)
    b = sv.submit(f, thr, descriptors=15)          # must wait for a's memory and slot
    with pytest.raises(ec.ECError) as e:
        sv.wait(b, timeout_ms=0)
    assert e.value.status == 6                     # EC_ERR_TIMEOUT from the bounded host wait
    ra, rb = sv.wait(a, 120000), sv.wait(b, 120000)
    np.testing.assert_array_equal(ra, rb)
    # a request that can never fit is refused at submission
    huge = np.zeros((600, 600, 600), np.uint8)
    with pytest.raises(ec.ECError) as e:
        sv.submit(huge, None, L=256, descriptors=1)
    assert e.value.status == 4
    # malformed request
    with pytest.raises(ec.ECError) as e:
        sv.submit(f, thr, descriptors=15, connectivity=8)
    assert e.value.status == 1
    sv.close()


def test_destroy_cancels_queued_requests(ctx):
    f, thr = workloads.config3(n=128, nblobs=30, L=200)
    f, thr = f.numpy(), thr.numpy()
    sv = ec.Server(device_mem_budget=64 << 20, max_slots=1, ctx=ctx)
    tickets = [sv.submit(f, thr, descriptors=1) for _ in range(6)]
    first = sv.result(tickets[0])
    sv.close()   # running work finishes, queued work is cancelled, nothing hangs
    assert sv.handle is None
    np.testing.assert_array_equal(first, oracle.ec_curves(f, thr, 200, 26, 1))
