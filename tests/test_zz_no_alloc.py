"""dem_mlp_loss_grad_noalloc (no device allocation, fixed scratch) gives the
results of dem_mlp_loss_grad.  Two calls in a row with different data show
that the accumulators are cleared between calls.  The file name sorts last so
that the check also runs after every other test has used the device."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_03445_gb300 as dem

    dem.load_library()
    return dem


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 6)).astype(np.float32)
    t = (np.sin(x[:, 0]) + 0.5 * x[:, 3] - 0.2 * x[:, 4] * x[:, 5]).astype(np.float32)
    return x, t


def _close(a, b, rel):
    return np.linalg.norm(a - b) <= rel * np.linalg.norm(b)


def test_matches_the_allocating_call_twice_in_a_row(dem):
    rng = np.random.default_rng(11)
    reg = dem.Regressor(params=(rng.normal(size=dem.capi.load().dem_mlp_num_params()) * 0.2)
                        .astype(np.float32))
    # the larger call first, so the second leaves stale rows past its end
    data = [_data(5000, 21), _data(1234, 22)]
    ref = [reg.loss_grad(x, t) for x, t in data]
    got = [reg.loss_grad_noalloc(x, t) for x, t in data]  # two calls in a row
    for (l_ref, g_ref), (l_na, g_na) in zip(ref, got):
        # same kernel, same inputs; only the order of the float atomics differs
        assert l_na == pytest.approx(l_ref, rel=1e-5)
        assert _close(g_na, g_ref, 1e-5)
    assert not _close(ref[0][1], ref[1][1], 1e-2)  # the two cases differ
    reg.close()


def test_rejects_more_rows_than_the_scratch(dem):
    from paper_2307_03445_gb300 import capi

    reg = dem.Regressor()
    n = capi.DEM_MLP_NOALLOC_MAX_ROWS + 1
    with pytest.raises(ValueError, match="fixed scratch"):
        reg.loss_grad_noalloc(np.zeros((n, 6), np.float32), np.zeros(n, np.float32))
    # the library refuses it too, before reading the (here one-row) arrays
    one = np.zeros(6, np.float32)
    loss = C.c_double()
    p = one.ctypes.data_as(C.POINTER(C.c_float))
    assert reg.lib.dem_mlp_loss_grad_noalloc(reg.h, n, p, p, C.byref(loss), None) == -3
    reg.close()
