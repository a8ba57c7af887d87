"""GPU tests of the batched form: many independent FP32 boxes advanced by one
persistent launch (or one launch per phase) per step.

Every box must come out identical to the same box advanced alone through
ch_step (same kernels, same arithmetic), and match the FP64 oracle within the
FP32 bar; the bounded grid barrier must report a timeout without hanging.
"""
import numpy as np
import pytest

from oracle import ch_oracle as co
from paper_2105_01865_gb300 import inputs, stability

from _parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2105_01865_gb300 import build, capi
    build.build()
    capi.load()


def small_boxes(seed=7):
    """Five boxes of different sizes, boundary conditions and parameters."""
    rng = np.random.default_rng(seed)
    specs = [((16, 16, 16), (0, 0, 0)), ((20, 12, 24), (0, 1, 0)), ((10, 18, 32), (1, 0, 1)),
             ((24, 24, 40), (0, 0, 1)), ((9, 11, 6), (1, 1, 1))]
    boxes = []
    for shape, bc in specs:
        nz, ny, nx = shape
        h = 1.0 / max(shape)
        cn = float(rng.uniform(0.5, 1.0)) * h
        pe = float(10 ** rng.uniform(2, 4))
        C = inputs.drops_field(shape, h, bc, [(nx * h * 0.5, ny * h * 0.45, nz * h * 0.55)], [0.3 * min(shape) * h],
                               cn)
        C = C + 0.02 * rng.standard_normal(shape)
        dt = 0.9 * stability.stable_dt(shape, h, bc, cn, pe)
        boxes.append(dict(shape=shape, h=h, bc=bc, cn=cn, pe=pe, C=C, dt=dt))
    return boxes


def single(box, nsteps):
    from paper_2105_01865_gb300.solver import Solver
    s = Solver(box["shape"], box["h"], box["bc"], box["cn"], box["pe"], box["dt"], box["C"], precision="f32")
    s.step(nsteps)
    out = s.field()
    s.close()
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_equals_single_box_runs(mode):
    from paper_2105_01865_gb300.solver import Batch
    boxes = small_boxes()
    b = Batch(boxes)
    b.set_schedule(mode, 2, 8, 1)
    b.step(4)
    got = b.fields()
    b.close()
    for box, g in zip(boxes, got):
        ref = single(box, 4)
        assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max(), box["shape"]


def test_batch_schedules_agree_bitwise():
    from paper_2105_01865_gb300.solver import Batch
    boxes = small_boxes(3)
    outs = []
    for sched in [(0, 1, 4, 0), (0, 2, 16, 1), (1, 3, 8, 1)]:
        b = Batch(boxes)
        b.set_schedule(*sched)
        b.step(3)
        outs.append(b.fields())
        b.close()
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(a, c)


def test_batch_matches_oracle_and_conserves_mass():
    from paper_2105_01865_gb300.solver import Batch
    boxes = small_boxes(11)
    b = Batch(boxes)
    m0 = b.mass()
    b.step(5)
    got = b.fields()
    m1 = b.mass()
    b.close()
    for box, g, a, c in zip(boxes, got, m0, m1):
        nz, ny, nx = box["shape"]
        p = co.Params(nx, ny, nz, box["h"], cn=box["cn"], pe=box["pe"], dt=box["dt"], bc=box["bc"])
        ref = co.step(box["C"], None, p, 5)
        assert_parity(g, ref, 1e-5, f"batched box {box['shape']}, 5 steps")
        assert abs(c - a) <= 1e-6 * abs(a)
        assert abs(a - co.mass(box["C"].astype(np.float32).astype(np.float64), p)) <= 1e-12 * abs(a) + 1e-15


def test_batch_barrier_timeout_is_reported_and_recoverable():
    """Poison the grid barrier (it expects one CTA more than launched): every
    wait expires after 20 ms, the kernel returns, ch_batch_sync reports
    CH_ETIMEOUT, and the batch works again afterwards."""
    from paper_2105_01865_gb300 import capi
    from paper_2105_01865_gb300.solver import Batch
    boxes = small_boxes(5)
    b = Batch(boxes)
    b.set_schedule(0, 1, 8, 1)
    capi.ch_batch_set_barrier_limit(b.handle, 20_000_000, 1)
    b.step(1)
    with pytest.raises(capi.CHError) as e:
        b.sync()
    assert e.value.status == capi.CH_ETIMEOUT
    capi.ch_batch_set_barrier_limit(b.handle, 2_000_000_000, 0)
    b.set_fields([box["C"] for box in boxes])
    b.step(2)
    b.sync()
    got = b.fields()
    b.close()
    for box, g in zip(boxes, got):
        ref = single(box, 2)
        assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max()


def test_batch_autotune_keeps_fields_and_results():
    from paper_2105_01865_gb300.solver import Batch
    boxes = small_boxes(13)
    b = Batch(boxes)
    report = b.autotune(1)
    assert "chosen:" in report
    b.step(2)
    got = b.fields()
    b.close()
    for box, g in zip(boxes, got):
        ref = single(box, 2)
        assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max()


def test_batch_64_uneven_boxes():
    """64 periodic boxes of 32^3..128^3 (uneven Cn, Pe, dt): mass per box and
    three sampled boxes against their single-box runs."""
    from paper_2105_01865_gb300.solver import Batch
    boxes = inputs.batch_boxes(64, seed=4)
    for box in boxes:
        box["dt"] = 0.9 * stability.stable_dt(box["shape"], box["h"], box["bc"], box["cn"], box["pe"])
    b = Batch(boxes)
    m0 = np.array(b.mass())
    b.step(3)
    m1 = np.array(b.mass())
    got = b.fields()
    b.close()
    assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0))
    for i in (0, 17, 63):
        ref = single(boxes[i], 3)
        assert np.abs(got[i] - ref).max() <= 1e-6 * np.abs(ref).max()
