"""The device-side failure path, made on purpose without faulting the GPU:
EC_OPT_TEST_GIVE_UP makes every block of the float32 TMA kernel give up its
first bounded wait at once (as if the staged plane had not arrived), while
the copies already requested still land before the block returns.  The
request must report EC_ERR_TIMEOUT (with validation on), its curves must
read INT64_MIN, and the context must stay usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_11740_gb300 import ec, workloads

pytestmark = pytest.mark.gpu

EC_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def ctx(libec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ec.Context(0)


def test_given_up_wait_poisons_curves_and_times_out(ctx):
    f, thr = workloads.config3(n=40, nblobs=10, L=65)
    fd, td = f.cuda(), thr.cuda()
    out = torch.zeros((3, 65), dtype=torch.int64, device="cuda")
    ctx.set_option(ec.EC_OPT_VALIDATE, 1)
    ctx.set_option(ec.EC_OPT_TEST_GIVE_UP, 1)
    try:
        with pytest.raises(ec.ECError) as e:
            ec.curve(fd, td, descriptors=13, out=out, ctx=ctx)
        assert e.value.status == EC_ERR_TIMEOUT
        torch.cuda.synchronize()
        assert bool(torch.all(out == torch.iinfo(torch.int64).min))
    finally:
        ctx.set_option(ec.EC_OPT_TEST_GIVE_UP, 0)
        ctx.set_option(ec.EC_OPT_VALIDATE, 0)
    # the context and the device are still usable
    got = ec.curve(fd, td, descriptors=13, ctx=ctx)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.ec_curves(f.numpy(), thr.numpy(), 65, 26, 13))
