"""The device input generators reproduce the host generators bit for bit."""
import numpy as np
import pytest

from gen import host as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gdev():
    from gen import device
    device.lib()
    return device


@pytest.mark.parametrize("variant", list("abcdef"))
def test_config2_device_equals_host(gdev, variant):
    n = (1 << 20) + 37
    d = gdev.config2(variant, n).cpu().numpy().view(np.uint32)
    assert np.array_equal(d, H.config2(variant, n))


def test_config1_and_config3_device_equals_host(gdev):
    assert np.array_equal(gdev.config1().cpu().numpy().view(np.uint32), H.config1())
    k, v = gdev.config3((1 << 20) + 11)
    hk, hv = H.config3((1 << 20) + 11)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), hk)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), hv)
