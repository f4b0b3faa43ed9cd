"""Checkpoint / resume: a run saved and resumed in a fresh handle continues
bitwise like the uninterrupted run, residual history included."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return dmrt


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_resume_is_bitwise_identical(dm, storage):
    grid, K = (20, 18, 16), 50
    a = dm.Cavity(grid, 1e5, wall_type=3, storage=storage, residual_interval=K)
    a.step(3 * K + 7)
    blob = a.save()
    a.step(4 * K)
    fa, ga = a.populations()
    ra = a.residual()
    b = dm.Cavity(grid, 1e5, wall_type=3, storage=storage, residual_interval=K)
    b.load(blob)
    assert b.params["steps"] == 3 * K + 7
    b.step(4 * K)
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert b.residual() == ra
    assert a.nusselt(0) == b.nusselt(0)


def test_checkpoint_of_another_cavity_is_rejected(dm):
    a = dm.Cavity((16, 16, 16), 1e5, wall_type=2)
    blob = a.save()
    for other in (dm.Cavity((16, 16, 16), 2e5, wall_type=2), dm.Cavity((16, 16, 16), 1e5, wall_type=1),
                  dm.Cavity((16, 16, 16), 1e5, wall_type=2, storage=1)):
        with pytest.raises(dm.DmrtError) as ei:
            other.load(blob)
        assert ei.value.status == dm.ERR_ARG
    with pytest.raises(dm.DmrtError):
        a.load(b"not a checkpoint" * 8)
