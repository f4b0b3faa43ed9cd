"""dmrt_nusselt_noalloc: Nusselt numbers without any device allocation.

Some callers may not allocate device memory once they are running (a host
application whose own memory pool owns the device memory, or a time-critical
loop where cudaMalloc / cudaFree would stall the device).  This entry point
keeps its scratch in a fixed array inside the library, so these tests check,
through the C ABI, that it gives the same numbers as dmrt_nusselt on two calls
in a row, and that it refuses sizes beyond its fixed limit.
"""

import ctypes

import pytest

pytestmark = pytest.mark.gpu

NU_RTOL = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return torch, dmrt


def _theta_on_device(torch, dmrt, cav):
    nx, ny, nz = cav.grid
    theta = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    dmrt.dmrt_fields(cav.h, theta=theta)
    return theta


def test_noalloc_matches_dmrt_nusselt_on_two_calls_in_a_row(env):
    torch, dmrt = env
    # the second cavity has fewer z rows, so stale rows of the first call
    # must not leak into the second result
    a = dmrt.Cavity((24, 20, 18), 1e5, wall_type=3)
    b = dmrt.Cavity((17, 12, 10), 3e4, wall_type=2)
    a.step(300)
    b.step(200)
    th_a = _theta_on_device(torch, dmrt, a)
    th_b = _theta_on_device(torch, dmrt, b)
    ref_a = a.nusselt(0)
    ref_b = b.nusselt(1)
    got_a = dmrt.dmrt_nusselt_noalloc(th_a, 0)
    got_b = dmrt.dmrt_nusselt_noalloc(th_b, 1)
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        for x, y in zip(got, ref):
            assert abs(x - y) <= NU_RTOL * abs(y), (got, ref)
    # repeating the first call after the second gives the first answer again
    again = dmrt.dmrt_nusselt_noalloc(th_a, 0)
    for x, y in zip(again, ref_a):
        assert abs(x - y) <= NU_RTOL * abs(y)


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    _, dmrt = env
    lib = dmrt.load()
    out = (ctypes.c_double * 3)()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.dmrt_nusselt_noalloc(fake, 8, 8, 8193, 0, None, out) == dmrt.ERR_ARG
    assert lib.dmrt_nusselt_noalloc(fake, 8, 1, 8, 0, None, out) == dmrt.ERR_ARG
    assert lib.dmrt_nusselt_noalloc(fake, 8, 8, 8, 2, None, out) == dmrt.ERR_ARG
    assert lib.dmrt_nusselt_noalloc(None, 8, 8, 8, 0, None, out) == dmrt.ERR_ARG


@pytest.mark.parametrize("nz,ny,nx,wall,on_stream", [(18, 12, 24, 0, False), (301, 4, 300, 1, True),
                                                     (9, 5, 257, 0, False)])
def test_noalloc_matches_the_oracle_on_a_seeded_field(env, nz, ny, nx, wall, on_stream):
    """The same seeded temperature field (rounded to float32, as the call
    reads it) through the allocation-free call and through the FP64 oracle's
    Nusselt numbers of a field: rows wider than one block's threads (nx >
    256) and more rows than the finishing block has threads (nz > 256) take
    the strided loops of both kernels; one case runs on a caller's stream."""
    import numpy as np

    import oracle
    from paper_1511_04633_gb300 import inputs

    torch, dmrt = env
    _, _, th = inputs.random_fields((nx, ny, nz), seed=70 + nz, dtheta=0.4)
    th32 = np.ascontiguousarray(th, dtype=np.float32)
    (r3, r2, rmax), _ = oracle.nusselt_from_theta(th32.astype(np.float64), wall)
    theta = torch.from_numpy(th32).cuda()
    stream = torch.cuda.Stream() if on_stream else None
    got = dmrt.dmrt_nusselt_noalloc(theta, wall, stream=stream)
    # FP64 local values of the same float32 inputs, summed in another order
    for x, y in zip(got, (r3, r2, rmax)):
        assert abs(x - y) <= 1e-12 * max(1.0, abs(y)), (got, (r3, r2, rmax))
