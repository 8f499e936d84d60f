"""The bounded mbarrier wait of the tensor-core kernels (kde_wait_probe): a
wait whose barrier is completed reports success; a wait on a barrier that
nothing ever completes gives up after its poll limit, the kernel ends and
reports it, and the context stays usable.  No fault, trap or hang is
involved: the wait simply runs out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import os

    from paper_1508_02766_gb300 import build, kde
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def test_completed_wait_reports_success(K):
    out = K.kde_wait_probe(True, 1 << 20).cpu().numpy()
    assert out[0] == 0


def test_wait_that_never_completes_gives_up_and_context_survives(K):
    limit = 1 << 14
    out = K.kde_wait_probe(False, limit).cpu().numpy()
    assert out[0] == 1
    assert out[1] > 0
    # the kernels' own limit (2^18 polls) must end in about a second: bound
    # it from the cycles this limit took (clocks of at least 1.4 GHz)
    seconds = out[1] / limit * (1 << 18) / 1.4e9
    assert seconds < 3.0, seconds
    # the context is still usable: a binning call after the timeout
    X = torch.rand(1000, 2, dtype=torch.float32, device="cuda")
    counts = K.kde_bin(X, (0.0, 0.0), (1.0, 1.0), (16, 16))
    torch.cuda.synchronize()
    assert int(counts.sum().item()) == 1000 * (1 << 32)


def test_rejects_bad_arguments(K):
    with pytest.raises(K.KDEError) as e:
        K.kde_wait_probe(True, 0)
    assert e.value.status == 1
