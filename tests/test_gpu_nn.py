"""Tensor-core (tcgen05) kernels of the bed surrogate against CPU references."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe
    L = swe.load_library()
    L.swe_nn_tc_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.swe_nn_tc_selftest.restype = ctypes.c_int
    return L


def _bf16(shape, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    t = torch.randn(*shape, generator=g).to(torch.bfloat16)
    return t, t.view(torch.int16).numpy().view(np.uint16).copy()


@pytest.mark.parametrize("n,k", [(32, 64), (16, 48), (32, 288 - 32)])
def test_tcgen05_gemm_matches_cpu(lib, n, k):
    """One 128 x n x k MMA chain through shared-memory descriptors and tensor
    memory equals the FP32 product of the same BF16 operands."""
    A, a = _bf16((128, k), 1)
    B, b = _bf16((n, k), 2)
    C = np.zeros((128, n), dtype=np.float32)
    st = lib.swe_nn_tc_selftest(n, k, a.ctypes.data, b.ctypes.data, C.ctypes.data)
    assert st == 0, st
    ref = (A.double() @ B.double().T).numpy()
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err


# ---------------------------------------------------------------- surrogate

def _bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _setup(seed, T=128, out_scale=1.0):
    import torch
    from oracle import cnn_oracle as C
    from paper_2103_15196_gb300 import swe
    S = swe.Surrogate(tile=T, max_batch=1, seed=seed)
    params = C.random_params(seed)
    params[5] = (params[5][0] * out_scale, params[5][1])
    for i, (Wm, b) in enumerate(params):
        S.set_params(i, Wm, b)
    # what the kernels see: BF16 weights, FP32 biases
    used = [(_bf16_round(Wm), np.asarray(b, np.float32).astype(np.float64)) for Wm, b in params]
    rng = np.random.default_rng(seed + 10)
    X = rng.normal(size=(T, T, 8))
    X[:, :, 7] = rng.random((T, T)) < 0.7          # activity mask
    Xb = _bf16_round(X)
    Xd = torch.from_numpy(Xb.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    return S, used, Xb, Xd


def test_surrogate_forward_matches_cpu_reference(lib):
    import torch
    from oracle import cnn_oracle as C
    T = 128
    S, used, Xb, Xd = _setup(3, T)
    out = torch.zeros((1, T, T), dtype=torch.float32, device="cuda")
    S.forward(Xd, out, 1)
    torch.cuda.synchronize()
    acts, ref = C.forward(Xb, used, round_fn=_bf16_round)
    got = out[0].cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 2e-2, rel
    S.close()


@pytest.mark.parametrize("kind", ["mse", "l1"])
def test_surrogate_gradients_match_cpu_reference(lib, kind):
    import torch
    from oracle import cnn_oracle as C
    T = 128
    S, used, Xb, Xd = _setup(4, T)
    S.set_loss(kind)
    rng = np.random.default_rng(40)
    target = rng.normal(size=(T, T)).astype(np.float32)
    td = torch.from_numpy(target).cuda()[None].contiguous()
    loss = S.train_step(Xd, td, 1, 1e-30)
    torch.cuda.synchronize()
    ref_loss, ref_grads, _ = C.loss_and_grads(Xb, target.astype(np.float64), used, round_fn=_bf16_round, loss=kind)
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    for layer in range(6):
        gW, gb = S.grads(layer)
        rW, rb = ref_grads[layer]
        eW = np.linalg.norm(gW - rW) / np.linalg.norm(rW)
        eb = np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-30)
        assert eW < 5e-2 and eb < 5e-2, (layer, eW, eb)
    S.close()


def test_surrogate_training_reduces_loss(lib):
    """A target the network can express (the masked linear extrapolation
    plus a blur of the bed channel): Adam on the tensor-core kernels must
    drive the loss down."""
    import torch
    T = 128
    S, used, Xb, Xd = _setup(5, T)
    b = Xb[:, :, 1]
    blur = 0.25 * (np.roll(b, 1, 0) + np.roll(b, -1, 0) + np.roll(b, 1, 1) + np.roll(b, -1, 1))
    tgt = Xb[:, :, 7] * (Xb[:, :, 6] + blur)
    td = torch.from_numpy(tgt.astype(np.float32)).cuda()[None].contiguous()
    losses = [S.train_step(Xd, td, 1, 2e-3) for _ in range(150)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
    S.close()


def _solver_case(swe, I):
    """A 256^2 flood scenario, spun up 60 steps so that sediment moves."""
    sc = I.ensemble_scenario(256, seed=901, manning=0.03, peak=300.0, d50_scale=1.0)
    Sv = swe.Solver(256, 256, 5.0, precision="fp32", A_J=0.01)
    Sv.set_manning(sc.manning, block=sc.manning_block)
    Sv.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
    Sv.set_state(sc.H, sc.Hu, sc.Hv, sc.b)
    Sv.run_steps(60)
    return sc, Sv


def test_surrogate_takeover_with_a_bad_network(lib):
    """A network that predicts a huge bed change fails its first judged
    window; the plain solver then runs every window, so the final state is
    bit-identical to a plain run of the same number of steps."""
    from paper_2103_15196_gb300 import inputs as I
    from paper_2103_15196_gb300 import swe
    sc, Sv = _solver_case(swe, I)
    S = swe.Surrogate(tile=128, max_batch=4, seed=9)
    Wm, b = S.params(5)
    S.set_params(5, Wm, b + 50.0)
    st = S.run(Sv, nwindows=4, K=20, f=5, judge_every=2, bound=0.02)
    assert st.judged == 1 and st.mode == 1 and st.takeover_window == 0
    assert st.plain_windows == 3 and st.surrogate_windows == 0 and st.err_max > 1.0
    got = Sv.get_state(np.float32)
    _, Ref = _solver_case(swe, I)
    Ref.run_steps(80)
    Ref.sync()
    for a, r in zip(got, Ref.get_state(np.float32)):
        assert np.array_equal(a, r)
    S.close()


def test_surrogate_windows_advance_the_bed_faster(lib):
    """A network whose last convolution is zero predicts the masked linear
    extrapolation of the window's first step: its judged error is the
    linear ablation's, surrogate windows advance the water K/f steps and
    the bed time f times as far, and set the bed to the window-start bed
    plus the first step's change times K."""
    import torch
    from paper_2103_15196_gb300 import inputs as I
    from paper_2103_15196_gb300 import swe
    K, f = 20, 5
    sc, Sv = _solver_case(swe, I)
    S = swe.Surrogate(tile=128, max_batch=4, seed=9)
    S.set_norm([0.0, 1.0, 0.0, 1.0, 1.0, 1.0, 1e-3, 1e-3 / K])
    Wm, b = S.params(5)
    S.set_params(5, 0 * Wm, 0 * b)
    st = S.run(Sv, nwindows=3, K=K, f=f, judge_every=3, bound=2.0)
    assert st.judged == 1 and st.surrogate_windows == 2 and st.mode == 0
    assert 0 < st.err_last < 1.0
    assert st.err_last == pytest.approx(st.err_linear_mean, rel=1e-12)
    assert st.bed_time > 1.8 * st.water_time
    # one more surrogate window by hand: save, one coupled step, apply
    b0 = Sv.get_state(np.float32)[3].astype(np.float64)
    S.save_bed(Sv)
    Sv.run_steps(1)
    b1 = Sv.get_state(np.float32)[3].astype(np.float64)
    S.apply(Sv)
    got = Sv.get_state(np.float32)[3].astype(np.float64)
    p = torch.tensor((b1 - b0) / (1e-3 / K)).to(torch.bfloat16).double().numpy()
    want = (b0 + p * 1e-3).astype(np.float32)
    assert np.allclose(got, want, rtol=0, atol=1e-6 * max(1.0, np.abs(b0).max()))
    S.close()


def test_surrogate_halo_tiles_match_the_whole_domain_network(lib):
    """The prediction of the surrogate windows runs the network only on the
    116^2 interior tiles that hold a cell of the activity mask, each as a
    128^2 image with a 6-cell margin (the receptive field of six 3x3
    layers).  On a 256^2 domain (ragged tiles) it must equal the same network
    run on the whole domain as one 256^2 image, cell by cell, with every
    inactive tile exactly unchanged."""
    import torch
    from oracle import cnn_oracle as C
    from paper_2103_15196_gb300 import inputs as I
    from paper_2103_15196_gb300 import swe
    sc, Sv = _solver_case(swe, I)
    n, K = 256, 50
    S = swe.Surrogate(tile=n, max_batch=1, seed=5)
    for i, (Wm, b) in enumerate(C.random_params(5)):
        S.set_params(i, Wm, b)
    H, _, _, b0 = Sv.get_state(np.float32)
    S.set_norm([float(H.mean()), float(H.std()) + 1e-6, float(b0.mean()), float(b0.std()) + 1e-6, 1.0, 1.0,
                1e-3, 1e-3 / K])
    S.save_bed(Sv)
    Sv.run_steps(1)
    X = torch.empty((1, n, n, 8), dtype=torch.bfloat16, device="cuda")
    assert S.pack_state(Sv, X) == 1
    out = torch.zeros((1, n, n), dtype=torch.float32, device="cuda")
    S.forward(X, out, 1)
    torch.cuda.synchronize()
    pred = out[0].cpu().numpy().astype(np.float64)
    mask = X[0, :, :, 7].float().cpu().numpy() > 0
    S.apply(Sv)
    got = Sv.get_state(np.float32)[3].astype(np.float64)
    want = b0.astype(np.float64) + pred * 1e-3
    assert np.abs(got - want).max() <= 2e-6 * max(1.0, np.abs(b0).max())
    # both branches are exercised: some interior tiles active, some not
    tiles = [(ty, tx) for ty in range(3) for tx in range(3)]
    act = [mask[ty * 116:(ty + 1) * 116, tx * 116:(tx + 1) * 116].any() for ty, tx in tiles]
    print("active interior tiles", act, "mask cells", int(mask.sum()))
    assert any(act) and not all(act), act
    for (ty, tx), a in zip(tiles, act):
        if not a:
            sl = (slice(ty * 116, (ty + 1) * 116), slice(tx * 116, (tx + 1) * 116))
            assert np.array_equal(got[sl], b0.astype(np.float64)[sl])
    S.close()
