"""Tensor-core kernels of the crater-surrogate MLP against the FP64 oracle.

The GEMM is compared with exact FP64 sums of the same BF16 products, on both of its
paths: operands gathered by threads (any strides) and operands streamed by TMA (K-major
rows of 16-byte multiples).  The network's
forward pass, gradient and Adam step are compared with the oracle in its BF16 form, which
rounds the same tensors to BF16 and does all arithmetic in FP64; the remaining differences
come from FP32 accumulation and FP32 GELU, which move a BF16 rounding of an activation or a
back-propagated gradient now and then by one unit (2^-8 relative) -- the tolerances below
allow for a fraction of those."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp_oracle as M
from paper_2403_04267_gb300 import salec, surrogate as S, workloads as W


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M_,N_,K_,at,bt", [
    (128, 256, 64, False, False),       # one full tile
    (1, 16, 1, False, False),           # smallest
    (300, 80, 200, False, False),       # ragged M tail, N not a multiple of 64, K tail
    (257, 300, 129, True, False),       # two N tiles, transposed A
    (130, 66, 520, False, True),        # transposed B
    (66, 5, 4096, True, True),          # weight-gradient shape: long K, tiny N
    (64, 256, 0, False, False),         # empty sum
    (257, 300, 256, False, False),      # K-major, 16-byte rows: TMA path, NT = 256 and a 44-row tail
    (512, 128, 1024, False, False),     # TMA path, 16 K slices through the 4-stage ring
    (4100, 66, 256, False, False),      # TMA path, many M tiles, N not a multiple of 16
])
def test_gemm_matches_exact_sums(M_, N_, K_, at, bt):
    rng = np.random.default_rng(M_ * 7 + N_ * 13 + K_)
    a = M.bf16_round(rng.standard_normal((M_, K_)))
    b = M.bf16_round(rng.standard_normal((N_, K_)))
    # stored transposed where asked: A(m, k) at k * M + m
    A = _bf16(a.T.copy() if at else a)
    B = _bf16(b.T.copy() if bt else b)
    a_str = (1, M_) if at else (K_, 1)
    b_str = (1, N_) if bt else (K_, 1)
    ldc = N_ + 3
    Cd = torch.full((max(M_, 1), ldc), float("nan"), dtype=torch.float32, device="cuda")
    S.gemm_bf16(M_, N_, K_, A, a_str, B, b_str, Cd, ldc)
    torch.cuda.synchronize()
    got = Cd.cpu().numpy().astype(np.float64)
    exact = a @ b.T
    bound = np.abs(a) @ np.abs(b).T
    err = np.abs(got[:M_, :N_] - exact)
    # FP32 accumulation of K products: far below 2^-14 of the sum of magnitudes
    assert np.all(err <= 2.0 ** -14 * bound + 1e-30), float(np.max(err / (bound + 1e-300)))
    assert np.all(np.isnan(got[:M_, N_:]))       # columns past N untouched


def _net(seed=11, gain=1.5):
    return W.mlp_init(seed, gain=gain).astype(np.float32).astype(np.float64)


def _data(B, seed=5):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    T = (0.5 * rng.standard_normal((B, 66))).astype(np.float32)
    return X, T


@pytest.mark.parametrize("B", [300, 1000, 1])
def test_forward_matches_oracle(B):
    """The inference pass (one fused kernel: five layers per 128-sample tile, activations
    kept on chip) against the oracle's BF16 form; ragged last tiles and a single sample."""
    theta = _net()
    X, _ = _data(B)
    net = S.MLP(1024)
    net.set_params(theta)
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref, _ = M.forward(theta, X.astype(np.float64), bf16=True)
    scale = np.max(np.abs(ref))
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-3
    assert np.max(np.abs(y - ref)) < 1e-2 * scale


def test_forward_inference_batch_sampled_rows():
    """The inference batch the benchmark times (65 536 draws), here with a ragged tail of 77
    more.  Rows are independent, so sampled rows (the first tile, the last two tiles and a
    random spread) are checked against the oracle one by one; every output is finite."""
    B = 65536 + 77
    theta = _net(seed=17)
    X, _ = _data(B, seed=9)
    net = S.MLP(B)
    net.set_params(theta)
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(y))
    rng = np.random.default_rng(4)
    rows = np.unique(np.concatenate([np.arange(128), np.arange(B - 205, B), rng.choice(B, 1500, replace=False)]))
    ref, _ = M.forward(theta, X[rows].astype(np.float64), bf16=True)
    assert np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref) < 1e-3
    assert np.max(np.abs(y[rows] - ref)) < 1e-2 * np.max(np.abs(ref))


def test_forward_rows_do_not_depend_on_the_batch():
    """Samples are independent: a sample's outputs are bitwise the same whether it is
    computed alone, in a 300-sample batch or in a 5000-sample batch (other tiles, other
    CTAs, the other slot of a tile pair)."""
    theta = _net(seed=19)
    X, _ = _data(5000, seed=10)
    net = S.MLP(5000)
    net.set_params(theta)
    Xd = torch.from_numpy(X).cuda()
    y_big = net.forward(Xd).cpu().numpy()
    y_mid = net.forward(Xd[:300].contiguous()).cpu().numpy()
    y_one = net.forward(Xd[257:258].contiguous()).cpu().numpy()
    assert np.array_equal(y_big[:300], y_mid)
    assert np.array_equal(y_big[257:258], y_one)


def test_gradient_is_deterministic():
    """The weight gradients split the batch over CTAs and add the partials in a fixed
    order, the bias gradients likewise: two evaluations agree bitwise."""
    theta = _net(seed=14)
    X, T = _data(3534, seed=8)
    net = S.MLP(3534)
    net.set_params(theta)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l1, g1 = net.gradient(Xd, Td)
    l2, g2 = net.gradient(Xd, Td)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    assert np.array_equal(g1, g2)
    assert np.all(np.isfinite(g1)) and np.any(g1 != 0.0)


def test_forward_single_chain():
    """One chain of units (input 0 -> 3 -> 7 -> 1 -> 250 -> output 65) with unit weights:
    output 65 is 2 gelu(gelu(gelu(gelu(x0)))) + 0.5 up to one BF16 rounding per layer and
    every other output is exactly 0."""
    theta = np.zeros(M.n_params())
    L = M.unpack(theta)
    L[0][0][3, 0] = 1.0
    L[1][0][7, 3] = 1.0
    L[2][0][1, 7] = 1.0
    L[3][0][250, 1] = 1.0
    L[4][0][65, 250] = 2.0
    L[4][1][65] = 0.5
    X = np.zeros((200, 5), dtype=np.float32)
    X[:, 0] = np.linspace(-2, 2, 200, dtype=np.float32)
    X[:, 3] = 9.0
    net = S.MLP(256)
    net.set_params(theta)
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    g = M.gelu
    expect = 2.0 * g(g(g(g(M.bf16_round(X[:, 0].astype(np.float64)))))) + 0.5
    assert np.max(np.abs(y[:, 65] - expect)) < 4 * 2.0 ** -8 * np.max(np.abs(expect))
    y[:, 65] = 0.0
    assert np.all(y == 0.0)


def test_gradient_matches_oracle():
    theta = _net(seed=12)
    X, T = _data(260, seed=6)
    net = S.MLP(512)
    net.set_params(theta)
    loss, g = net.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g = g.cpu().numpy().astype(np.float64)
    L_ref, g_ref = M.backward(theta, X.astype(np.float64), T.astype(np.float64), bf16=True)
    assert abs(loss - L_ref) <= 1e-4 * L_ref
    o = 0
    for l, (ni, no) in enumerate(zip(M.DIMS[:-1], M.DIMS[1:])):
        for name, cnt in (("W", ni * no), ("b", no)):
            a, r = g[o:o + cnt], g_ref[o:o + cnt]
            assert np.linalg.norm(a - r) <= 1e-2 * np.linalg.norm(r) + 1e-12, (l, name)
            o += cnt
    assert o == g.size


def test_adam_step_matches_oracle():
    theta = _net(seed=13)
    X, T = _data(128, seed=7)
    net = S.MLP(128)
    net.set_params(theta)
    lr = 1e-3
    net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), lr)
    got = net.get_params().astype(np.float64)
    _, g_ref = M.backward(theta, X.astype(np.float64), T.astype(np.float64), bf16=True)
    ref = theta.copy()
    M.adam(ref, g_ref, np.zeros_like(ref), np.zeros_like(ref), 1, lr)
    step_ref = ref - theta
    step = got - theta
    # the first Adam step is lr * g / (|g| + eps): +-lr wherever |g| >> eps; parameters
    # whose gradient sign is uncertain (|g| at rounding level) may move either way
    big = np.abs(g_ref) > 1e-3 * np.max(np.abs(g_ref))
    assert np.mean(np.abs(step[big] - step_ref[big]) < 1e-2 * lr) > 0.99
    assert np.max(np.abs(step)) <= lr * (1 + 1e-3)


def test_training_reduces_loss():
    rng = np.random.default_rng(21)
    X = rng.uniform(-1, 1, (1024, 5)).astype(np.float32)
    # a smooth target: each output a fixed combination of sines of the inputs
    Wt = rng.standard_normal((5, 66)) * 0.8
    T = np.sin(X.astype(np.float64) @ Wt).astype(np.float32)
    net = S.MLP(1024)
    net.set_params(W.mlp_init(3).astype(np.float32))
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0, _ = net.gradient(Xd, Td)
    for _ in range(300):
        net.train_step(Xd, Td, 2e-3)
    l1, _ = net.gradient(Xd, Td)
    net.check()
    assert l1 < 0.1 * l0, (l0, l1)


def test_multi_step_training_matches_single_steps():
    """salec_mlp_train: 60 steps as one call (one plain step, two 25-step graph replays, nine
    plain steps), learning rates from a device table, against 60 single-step calls with
    the same rates: the same arithmetic per step, the bias corrections formed on the device
    instead of the host (both in double precision)."""
    X, T = _data(700, seed=5)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    lr = S.cosine_lr(60, 2e-3)
    a = S.MLP(700)
    a.set_params(W.mlp_init(4).astype(np.float32))
    for k in range(60):
        a.train_step(Xd, Td, float(lr[k]))
    b = S.MLP(700)
    b.set_params(W.mlp_init(4).astype(np.float32))
    b.train(Xd, Td, torch.from_numpy(lr).cuda())
    pa, pb = a.get_params(), b.get_params()
    d = float(np.max(np.abs(pa - pb)) / np.max(np.abs(pa)))
    print("multi-step vs single steps: max parameter difference", d)
    assert d <= 1e-6
    # a second call continues the Adam step count
    b.train(Xd, Td, torch.from_numpy(lr[:30]).cuda())
    for k in range(30):
        a.train_step(Xd, Td, float(lr[k]))
    assert float(np.max(np.abs(a.get_params() - b.get_params())) / np.max(np.abs(pa))) <= 1e-6


def test_networks_on_separate_streams_train_as_alone():
    """Two networks trained at the same time on two streams end with the parameters each
    has when trained alone, bit for bit."""
    X, T = _data(900, seed=8)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    L = torch.from_numpy(S.cosine_lr(80, 2e-3)).cuda()
    alone = []
    for seed in (1, 2):
        n = S.MLP(900)
        n.set_params(W.mlp_init(seed).astype(np.float32))
        n.train(Xd, Td, L)
        alone.append(n.get_params())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    nets = []
    for seed, st in zip((1, 2), streams):
        n = S.MLP(900, stream=st)
        n.set_params(W.mlp_init(seed).astype(np.float32))
        nets.append(n)
    torch.cuda.synchronize()
    for n in nets:
        n.train(Xd, Td, L)
    for n, ref in zip(nets, alone):
        n.check()
        assert np.array_equal(n.get_params(), ref)


@pytest.mark.parametrize("members, batch", [(3, 900), (8, 200)])
def test_group_training_matches_members_trained_alone(members, batch):
    """salec_mlp_train_group: the members' GEMMs, Adam updates and step starts launched once
    for the whole group (80 steps: one plain step, three 25-step graph replays, four plain
    steps), with each member's plan and arithmetic as when trained alone: the same
    parameters bit for bit.  Batch 900 splits the weight gradients' K over CTAs (a
    deterministic partial sum per split), batch 200 does not."""
    X, T = _data(batch, seed=9)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    L = torch.from_numpy(S.cosine_lr(80, 2e-3)).cuda()
    alone = []
    for seed in range(members):
        n = S.MLP(batch)
        n.set_params(W.mlp_init(20 + seed).astype(np.float32))
        n.train(Xd, Td, L)
        alone.append(n.get_params())
    st = torch.cuda.Stream()
    nets = [S.MLP(batch, stream=st) for _ in range(members)]
    for seed, n in enumerate(nets):
        n.set_params(W.mlp_init(20 + seed).astype(np.float32))
    torch.cuda.synchronize()
    g = S.Group(nets, stream=st)
    g.train(Xd, Td, L)
    for n, ref in zip(nets, alone):
        n.check()
        assert np.array_equal(n.get_params(), ref)
    # a second call continues every member's Adam step count
    g.train(Xd, Td, L[:30])
    solo = S.MLP(batch)
    solo.set_params(W.mlp_init(20).astype(np.float32))
    solo.train(Xd, Td, L)
    solo.train(Xd, Td, L[:30])
    assert np.array_equal(nets[0].get_params(), solo.get_params())
