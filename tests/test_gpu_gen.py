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


def test_second_family_device_equals_host(gdev):
    for k in (10**2, 10**4, 10**6):
        n = 300_001
        d = gdev.gaussian_i32(n, 9, 40, k, start=17).cpu().numpy()
        assert np.array_equal(d, H.gaussian_i32(n, 9, 40, k, start=17)), k
    n = 200_003
    d = gdev.kmer_u64(n, 9, 50, start=123_456).cpu().numpy().view(np.uint64)
    assert np.array_equal(d, H.kmer_u64(n, 9, 50, start=123_456))
