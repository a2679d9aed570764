import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


class KernelBound:
    """The voxtet binding with the work distribution of the scanline step fixed: calls of the
    voxelize functions get ``kernel=K`` unless they pass one (1 = spans, 2 = slice units).
    GPU parity tests run once per distribution, since both must give the oracle's grid."""

    _BOUND = ("voxelize", "voxelize_fixed", "voxelize_grid", "voxelize_sparse")

    def __init__(self, module, kernel: int):
        self._m = module
        self.kernel = int(kernel)

    def __getattr__(self, name):
        a = getattr(self._m, name)
        if name in self._BOUND:
            def call(*args, **kw):
                kw.setdefault("kernel", self.kernel)
                return a(*args, **kw)
            return call
        return a


KERNELS = [1, 2]
KERNEL_IDS = ["spans", "slices"]
