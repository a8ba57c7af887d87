"""ch_mass_noalloc: the mass reduction for callers that cannot call cudaMalloc
(an application that owns the device memory budget through its own pool, or
a plug-in that is handed only pointers).  Its scratch is a fixed device array
inside the library.  Checked against the existing ch_mass entry point and
against the oracle's mass h^3 sum C (on the same values, in FP64), within the
FP64 parity tolerance the other tests use, on two calls in a row with
different grids, so a stale partial sum from the first call would show.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from oracle import ch_oracle as co

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2105_01865_gb300 import build, capi
    build.build()
    capi.load()


def _ch_mass(C0, h, prec):
    from paper_2105_01865_gb300.solver import Solver
    s = Solver(C0.shape, h, (0, 0, 1), 0.75 * h, 100.0, 1e-3, C0, precision=prec)
    m = s.mass()
    s.close()
    return m


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_mass_matches_ch_mass_twice(prec):
    from paper_2105_01865_gb300 import capi
    rng = np.random.default_rng(21)
    dtype = torch.float64 if prec == "f64" else torch.float32
    stream = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # first a larger grid, then a smaller one: the second call must not see
    # the first call's partial sums
    for shape, h in (((64, 48, 80), 1.0 / 64), ((9, 7, 11), 1.0 / 9)):
        C0 = 0.5 + 0.3 * rng.standard_normal(shape)
        if prec == "f32":
            C0 = C0.astype(np.float32).astype(np.float64)
        ref = _ch_mass(C0, h, prec)
        nz, ny, nx = shape
        ref_oracle = co.mass(C0, co.Params(nx, ny, nz, h, cn=0.75 * h, pe=100.0, dt=1e-3))
        C = torch.as_tensor(C0, dtype=dtype, device="cuda")
        stream.wait_stream(torch.cuda.current_stream())
        capi.ch_mass_noalloc(C, h, out, stream)
        stream.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (shape, got, ref)
        assert abs(got - ref_oracle) <= 1e-12 * abs(ref_oracle), (shape, got, ref_oracle)


def test_noalloc_rejects_grids_beyond_the_scratch_limit():
    from paper_2105_01865_gb300 import capi
    C = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = capi.load()
    import ctypes
    # 1024^3 cells > 65536 partials x 4096 cells: refused before any launch
    st = lib.ch_mass_noalloc(ctypes.c_void_p(C.data_ptr()), 1024, 1024, 1024, 1.0, capi.CH_F32,
                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert st == capi.CH_EINVAL


def test_noalloc_binding_refuses_bad_tensors_on_the_host():
    """The binding checks dtype, device, layout and the output before calling
    the library, so no launch ever reads past a buffer."""
    from paper_2105_01865_gb300 import capi
    stream = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    good = torch.zeros((5, 6, 7), dtype=torch.float32, device="cuda")
    for bad_C in (torch.zeros((5, 6, 7), dtype=torch.float16, device="cuda"),
                  torch.zeros((5, 6, 7), dtype=torch.int32, device="cuda"),
                  torch.zeros((5, 6, 14), dtype=torch.float32, device="cuda")[:, :, ::2],
                  torch.zeros((5, 6, 7), dtype=torch.float32)):
        with pytest.raises(ValueError):
            capi.ch_mass_noalloc(bad_C, 0.1, out, stream)
    for bad_out in (torch.zeros(1, dtype=torch.float32, device="cuda"), torch.zeros(1, dtype=torch.float64),
                    torch.zeros(0, dtype=torch.float64, device="cuda")):
        with pytest.raises(ValueError):
            capi.ch_mass_noalloc(good, 0.1, bad_out, stream)
