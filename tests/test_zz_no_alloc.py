"""qt_norm_static: the norm for callers that cannot let a library allocate
device memory (a process whose device memory all goes through its own
allocator or pool, or a latency-critical loop that cannot afford an
allocation).  It reduces amplitudes the caller already holds on the device,
into a double the caller holds on the device, with its partial sums in a
fixed file-scope device array instead of a cudaMalloc'd buffer.

The results are checked against qt_norm (the allocating entry point) on the
same states, on two calls in a row (the second call reuses the array the
first one left behind): bit for bit where both read the same bytes
(complex128, complex64), within 1e-12 for the float-float layout the test
rebuilds from the binary64 readout.  At n = 20 and 22 the reduction uses
all 1216 partial sums the array holds, each block striding over several
runs of the state.  This file sorts last so that a run stopping at the
first failure has run every other test before it; it also passes alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2210_01076_gb300 import binding as B
    from paper_2210_01076_gb300 import build as qbuild
    qbuild.build()
    B.load()
    return B


def _state(B, W, n, dtype):
    c = B.Circuit(n, dtype, min(n, 10))
    c.load_levels(W.random_circuit(n, 120, seed=n, p_multi=0.4))
    c.update_state()
    return c


@pytest.mark.parametrize("dtype", ["c128", "c64", "c128df"])
@pytest.mark.parametrize("n", [5, 17, 20, 22])
def test_norm_static_matches_qt_norm_twice(lib, dtype, n):
    import torch
    from paper_2210_01076_gb300 import workloads as W
    B = lib
    c = _state(B, W, n, dtype)
    want = c.norm()
    N = 1 << n
    if dtype == "c64":
        amps = torch.empty(N, dtype=torch.complex64, device="cuda")
        c.read_amplitudes_device(0, N, amps.data_ptr())
        code = B.QT_C64
    else:
        amps = torch.empty(N, dtype=torch.complex128, device="cuda")
        c.read_amplitudes_device(0, N, amps.data_ptr())
        code = B.QT_C128
        if dtype == "c128df":
            # the float-float layout: (re_hi, re_lo, im_hi, im_lo) per amplitude
            ri = torch.view_as_real(amps)
            hi = ri.to(torch.float32)
            lo = (ri - hi.to(torch.float64)).to(torch.float32)
            amps = torch.stack([hi[:, 0], lo[:, 0], hi[:, 1], lo[:, 1]], dim=1).contiguous()
            code = B.QT_C128_DF
    torch.cuda.synchronize()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(-1.0)
        B.qt_norm_static(amps.data_ptr(), N, code, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        if dtype == "c128df":
            assert abs(got - want) <= 1e-12, (got, want)
        else:
            # the same kernels with the same grid on the same bytes
            assert got == want, (got, want)
    c.close()


def test_norm_static_rejects_bad_arguments(lib):
    import torch
    B = lib
    buf = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cases = [
        ((buf.data_ptr(), 0, B.QT_C128, out.data_ptr()), B.QT_ERR_RANGE),
        ((buf.data_ptr(), (1 << 34) + 1, B.QT_C128, out.data_ptr()), B.QT_ERR_RANGE),
        ((0, 4, B.QT_C128, out.data_ptr()), B.QT_ERR_ARG),
        ((buf.data_ptr(), 4, B.QT_C128, 0), B.QT_ERR_ARG),
        ((buf.data_ptr(), 4, 9, out.data_ptr()), B.QT_ERR_ARG),
    ]
    for args, status in cases:
        with pytest.raises(B.QtError) as e:
            B.qt_norm_static(*args)
        assert e.value.status == status
        assert "qt_norm_static" in B.qt_last_error(None)
