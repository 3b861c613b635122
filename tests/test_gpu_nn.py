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
    extrapolation of the window's first two steps: its judged error is the
    linear ablation's, surrogate windows advance the water K/f steps and
    the bed time f times as far, and set the bed to the window-start bed
    plus the two steps' change times K/2."""
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
    # one more surrogate window by hand: save, two coupled steps, apply
    b0 = Sv.get_state(np.float32)[3].astype(np.float64)
    S.save_bed(Sv)
    Sv.run_steps(1)
    S.save_mid(Sv)
    Sv.run_steps(1)
    b2 = Sv.get_state(np.float32)[3].astype(np.float64)
    S.apply(Sv)
    got = Sv.get_state(np.float32)[3].astype(np.float64)
    p = torch.tensor(np.float32((b2 - b0).astype(np.float32) / np.float32(2 * 1e-3 / K))).to(torch.bfloat16).double().numpy()
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
    S.save_mid(Sv)
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


def test_trained_network_beats_the_linear_extrapolation_on_held_out_windows(lib):
    """What the learned part gains: trained on windows the solver itself
    generates (512^2 flood-channel scenarios of the benchmark's class, four
    256^2 tiles per window, K = 50 coupled steps), with the tensor-core
    forward and backward kernels and Adam, the network's relative L1 error of
    the window's bed change on held-out windows of an unseen scenario must be
    at most 0.9 x that of the linear extrapolation of the window's first two
    coupled steps (the network's own base, what the method without it would
    predict)."""
    import torch
    from paper_2103_15196_gb300 import inputs as I
    from paper_2103_15196_gb300 import swe
    n, T, K = 512, 256, 50

    def solver(seed):
        sc = I.ensemble_scenario(n, seed=seed, manning=0.035, peak=500.0, d50_scale=1.0)
        S = swe.Solver(n, n, 5.0, precision="fp32")
        S.set_manning(sc.manning, block=sc.manning_block)
        S.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
        S.set_state(*(a.astype(np.float32) for a in (sc.H, sc.Hu, sc.Hv, sc.b)))
        S.run_steps(300)
        return S

    # normalisation from one reference window (as the benchmark forms it)
    sv = solver(8100)
    H, Hu, Hv, b0 = sv.get_state(np.float32)
    sv.run_steps(K)
    db = (sv.get_state(np.float32)[3] - b0).astype(np.float64)
    sv.close()
    wet = H > 1e-4
    spd = np.sqrt(np.where(wet, Hu / np.maximum(H, 1e-4), 0) ** 2 + np.where(wet, Hv / np.maximum(H, 1e-4), 0) ** 2)
    vs = float(np.sqrt(np.mean(spd[wet] ** 2))) + 1e-6
    norm = [float(H.mean()), float(H.std()) + 1e-6, float(b0.mean()), float(b0.std()) + 1e-6,
            vs, vs ** 3, float(db.std()) + 1e-9, (float(db.std()) + 1e-9) / K]
    net = swe.Surrogate(tile=T, max_batch=4, seed=0)
    net.set_norm(norm)
    net.set_loss("l1")

    def windows(seed, count):
        X = torch.empty((4 * count, T, T, 8), dtype=torch.bfloat16, device="cuda")
        Y = torch.empty((4 * count, T, T), dtype=torch.float32, device="cuda")
        sv = solver(seed)
        for j in range(count):
            net.save_bed(sv)
            sv.run_steps(1)
            net.save_mid(sv)
            sv.run_steps(1)
            net.pack_state(sv, X[4 * j:4 * j + 4])
            sv.run_steps(K - 2)
            net.pack_target(sv, Y[4 * j:4 * j + 4])
            sv.run_steps(K)
        sv.close()
        return X, Y

    data = [windows(8200 + r, 30) for r in range(6)]
    X = torch.cat([d[0] for d in data])
    Y = torch.cat([d[1] for d in data])
    Xv, Yv = windows(8500, 10)
    nw = X.shape[0] // 4

    def held_out():
        out = torch.empty((4, T, T), dtype=torch.float32, device="cuda")
        e_net = e_lin = ref = 0.0
        for j in range(Xv.shape[0] // 4):
            net.forward(Xv[4 * j:4 * j + 4], out, 4)
            torch.cuda.synchronize()
            y = Yv[4 * j:4 * j + 4].double()
            lin = Xv[4 * j:4 * j + 4, :, :, 6].double() * Xv[4 * j:4 * j + 4, :, :, 7].double()
            e_net += float((out.double() - y).abs().sum())
            e_lin += float((lin - y).abs().sum())
            ref += float(y.abs().sum())
        return e_net / ref, e_lin / ref

    e0, lin = held_out()
    assert e0 == pytest.approx(lin, rel=1e-6)    # the untrained network is the extrapolation
    # a fixed number of steps and a step-based schedule (linear warm-up, then
    # a linear decay to a tenth): the kernels are deterministic, so is the run
    g = torch.Generator().manual_seed(0)
    total, warm, steps = 20000, 500, 0
    while steps < total:
        for i in torch.randperm(nw, generator=g).tolist():
            lr = 1e-3 * min(1.0, (steps + 1) / warm) * (0.1 + 0.9 * (1 - steps / total))
            net.train_step(X[4 * i:4 * i + 4], Y[4 * i:4 * i + 4], 4, lr)
            steps += 1
            if steps == total:
                break
    err, _ = held_out()
    net.close()
    print(f"held-out relative L1: network {err:.4f}, linear extrapolation {lin:.4f}, ratio {err / lin:.3f}, "
          f"{steps} training steps")
    assert err <= 0.9 * lin, (err, lin)
