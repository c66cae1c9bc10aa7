"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and its host FP64 weight routines agree with the oracle.
No GPU is touched."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kbe.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kbe_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def kbe():
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    return K


def test_every_declared_symbol_is_exported(kbe):
    lib = kbe.lib()
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_grid_weights_match_oracle(kbe):
    for seed in (0, 1, 2):
        t, order = W.grid(200, 0.02, 0.4, seed)
        for n in (0, 1, 2, 3, 7, 64, 199):
            a = kbe.grid_weights(t, order, n)
            b = oracle.composite_row(t, order, n)
            assert np.abs(a - b).max() < 1e-15 * 20 * max(1.0, np.abs(b).max()), (seed, n)


def test_grid_weights_high_orders(kbe):
    t, order = W.grid(80, 0.05, 0.3, 4, kmin=6, kmax=12)
    for n in (5, 13, 40, 79):
        a = kbe.grid_weights(t, order, n)
        b = oracle.composite_row(t, order, n)
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max(), n


def test_local_weights_adams_moulton(kbe):
    h = 0.25
    t = h * np.arange(8)
    w = kbe.local_weights(t[2:7], t[5], t[6])  # k = 4 over the last interval
    assert np.allclose(w / h, np.array([-19, 106, -264, 646, 251]) / 720.0, atol=1e-13, rtol=0)


def test_grid_validation_errors(kbe):
    t, order = W.grid(10, 0.1, 0.3, 0)
    bad = t.copy()
    bad[4] = bad[3]
    with pytest.raises(kbe.KBEError) as e:
        kbe.grid_weights(bad, order, 5)
    assert e.value.status == kbe.KBE_EINVAL
    o2 = order.copy()
    o2[3] = 13
    with pytest.raises(kbe.KBEError) as e:
        kbe.grid_weights(t, o2, 5)
    assert e.value.status == kbe.KBE_ERANGE
    o2[3] = 0
    with pytest.raises(kbe.KBEError) as e:
        kbe.grid_weights(t, o2, 5)
    assert e.value.status == kbe.KBE_ERANGE
    t2 = t.copy()
    t2[0] = 0.1
    with pytest.raises(kbe.KBEError) as e:
        kbe.grid_weights(t2, order, 5)
    assert e.value.status == kbe.KBE_EINVAL
    with pytest.raises(kbe.KBEError):
        kbe.grid_weights(t, order, 10)  # n outside [0, n_t)
    with pytest.raises(kbe.KBEError):
        kbe.local_weights(np.array([0.0, 1.0, 1.0]), 1.0, 2.0)  # repeated node


def test_create_rejects_bad_sizes_without_touching_the_gpu(kbe):
    lib = kbe.lib()
    h = ctypes.c_void_p()
    assert lib.kbe_create(0, 10, ctypes.byref(h)) == kbe.KBE_EINVAL
    assert lib.kbe_create(65, 10, ctypes.byref(h)) == kbe.KBE_EINVAL
    assert lib.kbe_create(4, 0, ctypes.byref(h)) == kbe.KBE_EINVAL
    assert lib.kbe_create(4, 10, None) == kbe.KBE_EINVAL
    assert b"norb" in lib.kbe_last_error(None) or b"NULL" in lib.kbe_last_error(None)
    # calls on a NULL context are rejected
    assert lib.kbe_history_slice(None, 0, 0, None, None, None, None, None, None) == kbe.KBE_EINVAL
    assert lib.kbe_debug_withhold_run(None, 0, 1) == kbe.KBE_EINVAL
    assert lib.kbe_run_steps(None, 1, 1, 2, 0, None, None, None, None, None, None, None) == kbe.KBE_EINVAL
    assert lib.kbe_destroy(None) == kbe.KBE_OK
