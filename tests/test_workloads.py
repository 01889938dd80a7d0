"""The seeded generators (CPU only): the torch generators used for inputs
too large to generate on the host give the numpy generators' exact bits, so
the benchmark's device-generated inputs are the same workloads the tests and
the oracle use."""
import numpy as np
import pytest

from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,seed", [(1, 5), (1000, 77), ((1 << 20) + 3, W.DEFAULT_SEED),
                                    ((1 << 26) + 5, 0xB5EED001)])
def test_torch_generators_match_numpy(n, seed):
    a = W.uniform_int32(n, seed)
    b = W.uniform_int32_torch(n, seed, device="cpu").numpy()
    assert np.array_equal(a, b)
    if n <= (1 << 20) + 3:
        a = W.uniform_uint64(n, seed)
        b = W.uniform_uint64_torch(n, seed, device="cpu").numpy().view(np.uint64)
        assert np.array_equal(a, b)


def test_splitmix64_reference_values():
    # splitmix64 with state 0: the first outputs of the published generator
    # (Steele, Lea & Flood 2014; Vigna's reference implementation), i.e.
    # element i of stream 0 is mix(0 + (i + 1) * golden)
    got = W.splitmix64(0, 0, 3)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    t = W.splitmix64_torch(0, 0, 3, device="cpu").numpy().view(np.uint64)
    assert np.array_equal(got, t)


@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "dup16"])
@pytest.mark.parametrize("n", [1, 1000, (1 << 20) + 7])
def test_torch_int32_distributions_match_numpy(dist, n):
    a = W.int32_keys(dist, n, seed=0xB5EED005)
    b = W.int32_keys_torch(dist, n, seed=0xB5EED005, device="cpu").numpy()
    assert np.array_equal(a, b)
