"""What the learned warm start gains over the method without it.

The surrogate network only initialises a cavity; the lattice Boltzmann
solve then runs to its own convergence criterion and decides the answer.
These tests measure, on cavities the network never trained on, the steps
until the hot-wall Nu_3D (Eqs. (39)-(40)) stays within 1e-3 of a tighter
from-rest reference (the solve continued to residual < 1e-9), once from rest
and once from the network's prediction, and assert that the warm start
needs fewer steps and ends at the same Nu.

* A network trained inside the test, from scratch, on steady states that
  the library's ensemble solver generates at 32^3 (the whole pipeline:
  data, training by the library's own kernels, warm start).
* The shipped network (``weights/warm_start_64cube.npz``, trained on 512
  steady states at 64^3 by ``python -m paper_1511_04633_gb300.surrogate
  --save-params``), on held-out draws at 64^3 and at 128^3.
"""

import pytest

from paper_1511_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

NU_RTOL = 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    from paper_1511_04633_gb300 import surrogate as S
    dmrt.load()
    return torch, dmrt, S


def _assert_gain(r):
    cold, warm = r["from_rest"], r["warm"]
    assert cold["steps_to_nu"] is not None and warm["steps_to_nu"] is not None, r
    assert warm["steps_to_nu"] < cold["steps_to_nu"], r
    # equal accuracy: the warm-started solve converges to the same Nu
    assert r["nu_rel_diff"] <= NU_RTOL, r


def test_network_trained_here_gains_on_held_out_cavities(env):
    torch, dm, S = env
    n = 32
    draws = inputs.ensemble_draws(42, seed=77, edges=(n,), log10_ra=(3.0, 5.0))
    train, held_out = draws[:40], draws[40:]
    ra, wall, tgt, info = S.steady_dataset(n, train, tol=1e-6, max_steps=100_000)
    assert info["converged"] == len(train), info
    sur = dm.Surrogate(n, 2, (16, 32, 64), storage=dm.STORE_BF16, max_batch=4, seed=3)
    hist = S.train(sur, ra, wall, tgt, epochs=60, batch=4, lr=2e-3, seed=1)
    assert len(hist) == 60 and hist[-1] < 0.05 * hist[0], hist
    for d in held_out:
        _assert_gain(S.compare_warm_start(sur, n, d["Ra"], d["wall"], tol=1e-7, nu_rtol=NU_RTOL))


@pytest.mark.parametrize("grid,index", [(64, 0), (64, 7), (128, 2)])
def test_shipped_network_gains_on_held_out_cavities(env, grid, index):
    torch, dm, S = env
    sur, info = S.load_surrogate()
    assert info["train"] == S.TRAIN_COUNT and info["seed"] == S.TRAIN_SEED
    d = S.held_out_draws(index + 1)[index]
    _assert_gain(S.compare_warm_start(sur, grid, d["Ra"], d["wall"], tol=1e-7, nu_rtol=NU_RTOL))
