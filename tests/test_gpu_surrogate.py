"""The warm-start surrogate's CUDA forward and backward passes against the
FP64 numpy oracle of the same network, its training, and its warm start."""

import numpy as np
import pytest

import oracle
from oracle import surrogate as S
from paper_1511_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

CFG = dict(grid=16, depth=1, channels=(8, 16))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return torch, dmrt


def _setup(dm, storage, seed=5, scale=0.3):
    sur = dm.Surrogate(CFG["grid"], CFG["depth"], CFG["channels"], storage=storage, max_batch=2)
    net = S.UNet(CFG["grid"], CFG["depth"], CFG["channels"])
    assert sur.param_count == net.count
    p = inputs.random_weights(net.count, seed=seed, scale=scale)
    sur.set_params(p)
    return sur, net, p


def test_forward_matches_the_oracle_fp32(env):
    torch, dm = env
    sur, net, p = _setup(dm, dm.STORE_F32)
    ra, wall = [2e3, 3e5], [1, 3]
    got = sur.predict(ra, wall)
    ref, _ = net.forward(p.astype(np.float64), S.features(ra, wall, CFG["grid"]))
    ref = ref.reshape(2, -1, 5)
    assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_gradients_match_the_oracle_fp32(env):
    torch, dm = env
    sur, net, p = _setup(dm, dm.STORE_F32)
    ra, wall = [5e3, 8e4], [2, 1]
    n = CFG["grid"]
    t = inputs.random_targets((2, n, n, n, 5), seed=9)
    g_gpu, loss_gpu = sur.gradients(ra, wall, torch.from_numpy(t.reshape(2, -1, 5)).cuda())
    loss_ref, g_ref = net.loss_and_grad(p.astype(np.float64), S.features(ra, wall, n), t.astype(np.float64))
    assert abs(loss_gpu - loss_ref) <= 1e-5 * loss_ref
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-4, rel
    # every layer, not just the largest
    for (wo, bo), (cin, cout, k, _) in zip(net.offsets, net.layers):
        seg = slice(wo, bo + cout)
        r = np.linalg.norm(g_gpu[seg] - g_ref[seg]) / max(np.linalg.norm(g_ref[seg]), 1e-30)
        assert r <= 1e-3, (cin, cout, k, r)


def test_bf16_storage_tracks_the_oracle(env):
    torch, dm = env
    sur, net, p = _setup(dm, dm.STORE_BF16)
    ra, wall = [5e3, 8e4], [2, 1]
    n = CFG["grid"]
    got = sur.predict(ra, wall)
    pb = torch.from_numpy(p).to(torch.bfloat16).float().numpy().astype(np.float64)
    ref, _ = net.forward(pb, S.features(ra, wall, n))
    ref = ref.reshape(2, -1, 5)
    assert np.abs(got - ref).max() <= 5e-2 * np.abs(ref).max()
    t = inputs.random_targets((2, n, n, n, 5), seed=9)
    g_gpu, _ = sur.gradients(ra, wall, torch.from_numpy(t.reshape(2, -1, 5)).cuda())
    _, g_ref = net.loss_and_grad(pb, S.features(ra, wall, n), t.astype(np.float64))
    cos = float(np.dot(g_gpu, g_ref) / (np.linalg.norm(g_gpu) * np.linalg.norm(g_ref)))
    assert cos >= 0.99, cos


@pytest.mark.parametrize("k,cin,cout", [(3, 16, 32), (3, 8, 16), (3, 32, 5), (1, 16, 5), (3, 128, 64)])
@pytest.mark.parametrize("out_f32", [False, True])
def test_tensor_core_convolution_matches_the_definition(env, k, cin, cout, out_f32):
    """The bf16 tensor-core convolution on values exactly representable in
    bf16 against the oracle's FP64 convolution: only the FP32 accumulation
    and (for bf16 output) the final rounding differ."""
    torch, dm = env
    n, batch = 16, 2
    x = torch.from_numpy(inputs.random_targets((batch, n, n, n, cin), seed=21)).to(torch.bfloat16)
    w = torch.from_numpy(inputs.random_weights(k ** 3 * cout * cin, seed=22, scale=0.2)).to(torch.bfloat16)
    b = torch.from_numpy(inputs.random_weights(cout, seed=23, scale=0.5))
    y = torch.empty((batch, n, n, n, cout), dtype=torch.float32 if out_f32 else torch.bfloat16, device="cuda")
    dm.dmrt_nn_conv3d(x.cuda(), w.cuda(), b.cuda(), y, batch, n, cin, cout, k, act=1)
    assert dm.dmrt_nn_tensor_core_errors(reset=True) == 0
    ref = S.leaky(S.conv3d(x.double().numpy(), w.double().numpy().reshape(k ** 3, cout, cin), b.double().numpy(), k))
    got = y.double().cpu().numpy()
    scale = np.abs(ref).max()
    tol = 2e-5 if out_f32 else 8e-3
    assert np.abs(got - ref).max() <= tol * scale


def test_training_overfits_a_batch_and_is_repeatable(env):
    """The student (zero output head) learns the outputs of a teacher network
    with random weights; two runs from the same seed are bitwise equal."""
    torch, dm = env
    ra, wall = [3e3, 2e5], [2, 3]
    teacher = dm.Surrogate(CFG["grid"], CFG["depth"], CFG["channels"], storage=dm.STORE_F32, max_batch=2)
    teacher.set_params(inputs.random_weights(teacher.param_count, seed=12, scale=0.2))
    t = torch.from_numpy(teacher.predict(ra, wall)).cuda()
    runs = []
    for _ in range(2):
        sur = dm.Surrogate(CFG["grid"], CFG["depth"], CFG["channels"], storage=dm.STORE_BF16,
                           max_batch=2, seed=3)
        losses = [sur.train_step(ra, wall, t, 2e-3) for _ in range(120)]
        runs.append((losses, sur.params()))
    assert runs[0][0][-1] < 0.3 * runs[0][0][0]
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("N,wall,Ra", [(24, 1, 3e4), (12, 3, 5e5), (16, 2, 2e3)])
def test_warm_start_matches_the_oracle_mapping(env, N, wall, Ra):
    """dmrt_warm_start against the oracle's chain on a network with random
    weights (so the prediction varies along every axis and channel): the
    FP64 network forward, trilinear resampling between the cell-centred grids
    (16^3 to N^3: up by 3/2, down by 3/4, and the identity), the channel
    scalings and the equilibrium initialisation, compared through the
    fields of the pulled populations.  A wrong interpolation weight, axis
    order, cell-centre offset or channel-to-field assignment fails."""
    torch, dm = env
    # weights of scale 0.12 give outputs of order 0.1-0.3: velocities near
    # 0.01, as in a converged cavity
    sur, net, p = _setup(dm, dm.STORE_F32, seed=17, scale=0.12)
    cav = dm.Cavity((N, N, N), Ra, wall_type=wall)
    sur.warm_start(cav, Ra, wall)
    rho, u, th = cav.fields()
    pred, _ = net.forward(p.astype(np.float64), S.features([Ra], [wall], CFG["grid"]))
    uc = np.sqrt(cav.params["gbeta"] * N)
    r0, u0, t0 = S.warm_start_fields(pred[0], N, uc)
    # the prediction must vary, or the comparison could not see a resampling error
    assert np.ptp(t0) > 0.1 * np.abs(t0).max() and np.ptp(u0[0]) > 0.1 * np.abs(u0[0]).max()
    o = oracle.Oracle.physical((N, N, N), wall, Ra)
    o.init_fields(r0, u0, t0)
    ro, uo, to = o.fields()
    o.close()
    # FP32 network (checked to 1e-4 of its output scale above) and FP32 fields
    tol = 2e-4
    assert np.abs(th - to).max() <= tol * np.abs(to).max()
    assert np.abs(u - uo).max() <= tol * np.abs(uo).max()
    assert np.abs(rho - ro).max() <= tol * np.abs(ro - 1).max() + 1e-6


def test_surrogate_rejects_bad_configurations(env):
    torch, dm = env
    for grid, depth, ch in ((20, 1, (8, 16)), (16, 2, (8, 16, 32)), (16, 1, (12, 16))):
        with pytest.raises(dm.DmrtError):
            dm.Surrogate(grid, depth, ch)


@pytest.mark.parametrize("channels", [(16, 32), (8, 16)])
def test_bf16_gradients_per_layer(env, channels):
    """The bf16 path (tensor-core convolutions, weight gradients over all 27
    taps per block) against the FP64 oracle evaluated at the bf16-rounded
    parameters, layer by layer: the gradients may differ only by the bf16
    rounding of activations and output gradients."""
    torch, dm = env
    n = 16
    sur = dm.Surrogate(n, 1, channels, storage=dm.STORE_BF16, max_batch=2)
    net = S.UNet(n, 1, channels)
    p = inputs.random_weights(net.count, seed=31, scale=0.3)
    sur.set_params(p)
    pb = torch.from_numpy(p).to(torch.bfloat16).float().numpy().astype(np.float64)
    ra, wall = [4e3, 6e5], [3, 2]
    t = inputs.random_targets((2, n, n, n, 5), seed=32)
    g_gpu, _ = sur.gradients(ra, wall, torch.from_numpy(t.reshape(2, -1, 5)).cuda())
    _, g_ref = net.loss_and_grad(pb, S.features(ra, wall, n), t.astype(np.float64))
    for (wo, bo), (cin, cout, k, _) in zip(net.offsets, net.layers):
        seg = slice(wo, bo)  # weights
        a, b = g_gpu[seg], g_ref[seg]
        cos = float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert cos >= 0.995 and rel <= 5e-2, (cin, cout, k, cos, rel)


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 32), (8, 32)])
@pytest.mark.parametrize("out_f32", [False, True])
def test_tensor_core_convolution_on_a_64_grid(env, cin, cout, out_f32):
    """The tcgen05 convolution streamed along z (runs of 7 planes and a last
    run of one on a 64^3 grid) against the definition."""
    torch, dm = env
    n, batch, k = 64, 1, 3
    x = torch.from_numpy(inputs.random_targets((batch, n, n, n, cin), seed=41)).to(torch.bfloat16)
    w = torch.from_numpy(inputs.random_weights(k ** 3 * cout * cin, seed=42, scale=0.2)).to(torch.bfloat16)
    b = torch.from_numpy(inputs.random_weights(cout, seed=43, scale=0.5))
    y = torch.empty((batch, n, n, n, cout), dtype=torch.float32 if out_f32 else torch.bfloat16, device="cuda")
    dm.dmrt_nn_conv3d(x.cuda(), w.cuda(), b.cuda(), y, batch, n, cin, cout, k, act=1)
    assert dm.dmrt_nn_tensor_core_errors(reset=True) == 0
    ref = S.leaky(S.conv3d(x.double().numpy(), w.double().numpy().reshape(k ** 3, cout, cin), b.double().numpy(), k))
    got = y.double().cpu().numpy()
    tol = 2e-5 if out_f32 else 8e-3
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_channel_blocks_of_the_small_grid_convolution_give_the_same_bits(env):
    """At 8^3 the mma.sync convolution takes 16 output channels per block
    when 32 per block would leave most SMs idle (a small batch), and 32 per
    block otherwise (a large batch).  Every output accumulates the same MMAs
    in the same order either way: the first samples of a large batch come out
    bitwise equal to the same samples alone, and both match the definition."""
    torch, dm = env
    n, cin, cout, big = 8, 64, 128, 64
    x = torch.from_numpy(inputs.random_targets((big, n, n, n, cin), seed=41)).to(torch.bfloat16).cuda()
    w = torch.from_numpy(inputs.random_weights(27 * cout * cin, seed=42, scale=0.2)).to(torch.bfloat16).cuda()
    b = torch.from_numpy(inputs.random_weights(cout, seed=43, scale=0.5)).cuda()
    y_small = torch.empty((2, n, n, n, cout), dtype=torch.float32, device="cuda")
    y_big = torch.empty((big, n, n, n, cout), dtype=torch.float32, device="cuda")
    dm.dmrt_nn_conv3d(x[:2].contiguous(), w, b, y_small, 2, n, cin, cout, 3, act=1)
    dm.dmrt_nn_conv3d(x, w, b, y_big, big, n, cin, cout, 3, act=1)
    torch.cuda.synchronize()
    assert torch.equal(y_small, y_big[:2])
    xs = x[:2].double().cpu().numpy()
    ref = S.leaky(S.conv3d(xs, w.double().cpu().numpy().reshape(27, cout, cin), b.double().cpu().numpy(), 3))
    got = y_small.double().cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
