"""The double-float arithmetic the recursion's scores use (log-likelihood and
transition terms evaluated on the FP32 pipe as pairs of FP32 numbers, about
48 bits) against numpy's float64 exp, log and sqrt on the same inputs. The
inputs are float64 values; the device splits each into an FP32 pair, which
carries all but the last ~5 of its 53 bits, so the comparison is against the
function of that pair: relative 2^-44 for exp and sqrt, absolute 2^-45
(times max(1, |log x|)) for log. exp is held on |x| < 60: further out the
low FP32 part of the result leaves the normal range (the recursion uses
exp on [-45, 0])."""
import numpy as np
import pytest

from paper_2312_08684_gb300 import _binding as abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def _pair(x):
    """The value the device sees: the FP32 pair (hi, lo) of each input, summed in float64."""
    hi = x.astype(np.float32).astype(np.float64)
    lo = (x - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def test_exp():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-45.0, 0.0, 20000), rng.uniform(-60.0, 60.0, 5000),
                        [0.0, -1e-12, 1e-12, -0.3465735902799727, 0.3465735902799727, -45.0]])
    got = abi.smap_debug_df(0, x)
    ref = np.exp(_pair(x))
    assert np.all(np.abs(got - ref) <= 2.0 ** -44 * ref)
    assert abi.smap_debug_df(0, np.zeros(1))[0] == 1.0


def test_log():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(1.0, 12.0, 20000), np.exp(rng.uniform(-30.0, 30.0, 5000)),
                        [1.0, 1.0 + 2.0 ** -40, 2.0, np.sqrt(2.0), 0.5, 11.999]])
    got = abi.smap_debug_df(1, x)
    ref = np.log(_pair(x))
    assert np.all(np.abs(got - ref) <= 2.0 ** -45 * np.maximum(1.0, np.abs(ref)))
    assert abi.smap_debug_df(1, np.ones(1))[0] == 0.0


def test_sqrt():
    rng = np.random.default_rng(3)
    x = np.concatenate([np.exp(rng.uniform(-20.0, 20.0, 20000)), rng.uniform(0.0, 2e4, 5000), [1.0, 2.0, 1e-6]])
    x = x[x > 0]
    got = abi.smap_debug_df(2, x)
    ref = np.sqrt(_pair(x))
    assert np.all(np.abs(got - ref) <= 2.0 ** -44 * ref)
