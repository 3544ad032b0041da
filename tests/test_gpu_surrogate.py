"""The learned warm start on the GPU: its network against the FP64 reference
(oracle/mlp.py, same BF16 rounding points), its training, and the
warm-started solve against the FP64 oracle of the update itself."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2407_18304_gb300 import rhd, surrogate, synth
from parity import MAX_UNCONVERGED, agreed, conservation, converged, errors, run_oracle, select

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
TIGHT = dict(tol=1e-14, tol_outer=1e-15)
FLOOR = 10 * TIGHT["tol"] / FP64_TOL
MIXED_BOUND = 1e-6
DEFAULT_FLOOR = 10 * 1e-11 / MIXED_BOUND


def _random_net(G, seed):
    sur = rhd.Surrogate(G, seed)
    rng = np.random.default_rng(seed)
    nin, nout = sur.n_features, sur.n_outputs
    p = M.init_params(nin, nout, seed).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, nin), rng.uniform(0.5, 2, nin),
                           rng.normal(0, 1, nout), rng.uniform(0.5, 2, nout)]).astype(np.float32)
    sur.set_params(torch.tensor(p, device="cuda"), torch.tensor(norm, device="cuda"))
    return sur, p.astype(np.float64), norm.astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("G,n", [(4, 1000 + 37), (16, 300), (32, 129), (64, 777)])
def test_forward_matches_the_reference_network(G, n):
    sur, p, norm = _random_net(G, 11 + G)
    rng = np.random.default_rng(G)
    x = rng.normal(0, 1.5, (n, sur.n_features)).astype(np.float32)
    y = sur.predict(torch.tensor(x, device="cuda")).cpu().numpy().astype(np.float64)
    ref = M.predict(p, norm, x.astype(np.float64), sur.n_features, sur.n_outputs, bf=True)
    ref64 = M.predict(p, norm, x.astype(np.float64), sur.n_features, sur.n_outputs, bf=False)
    e, e64 = _rel(y, ref), _rel(y, ref64)
    print(f"G={G} forward rel error vs BF16 reference {e:.2e}, vs FP64 {e64:.2e}")
    assert e < 1e-2 and e64 < 3e-2
    assert sur.error_flag() == 0


@pytest.mark.parametrize("G,n", [(4, 1000 + 37), (16, 300), (33, 129), (64, 777)])
def test_fused_warm_start_matches_the_network(G, n):
    """The fused inference kernel (features, four layers on chip, Newton
    start) against the same network through rhd_surrogate_features +
    rhd_surrogate_predict and the warm-start formulas written out here:
    E_int,0 = rho c_v T exp(y_T), R_g,0 / E_tot = (E_g / E_tot) expm1(y_g) - S_g / E_tot,
    both outputs held to [-5, 5] and [-30, 30].  Ragged last tile (n not a
    multiple of 128), a source term, and group counts whose feature and
    output widths are not multiples of 16."""
    sur, p, norm = _random_net(G, 70 + G)
    w = synth.preset("mixed_128cube_ng16", n_cells=n, seed=90 + G, n_groups=G, device="cuda")
    w.state["src"] = 0.1 * w.state["erad"].flip(0).contiguous()
    kw = dict(dt=w.dt, c_v=w.c_v, consts=w.consts)
    eint, r = sur.warm_start(w.state, w.edges, w.law, **kw)
    x = sur.features(w.state, w.edges, w.law, **kw)
    y = sur.predict(x).cpu().numpy().astype(np.float64)
    st = synth.to_numpy(w.state)
    ke = 0.5 * (st["mom"] ** 2).sum(0) / st["rho"]
    T = (st["egas"] - ke) / (st["rho"] * w.c_v)
    etot = st["egas"] + (st["erad"] + st["src"]).sum(0) * w.consts["c"] / w.consts["c_hat"]
    eint_ref = st["rho"] * w.c_v * T * np.exp(np.clip(y[:, 0], -5, 5))
    yg = np.clip(y[:, 1:].T, -30, 30)
    r_ref = st["erad"] / etot * np.expm1(yg) - st["src"] / etot
    e1 = np.max(np.abs(eint.cpu().numpy() / eint_ref - 1))
    # R_g is formed in FP32 from two terms: measure against their size
    scale = st["erad"] / etot * (1 + np.abs(np.expm1(yg))) + st["src"] / etot
    e2 = np.max(np.abs(r.cpu().numpy() - r_ref) / scale)
    print(f"G={G} fused warm start vs network: E_int {e1:.2e}, R_g {e2:.2e}")
    assert e1 < 1e-5 and e2 < 1e-5
    assert sur.error_flag() == 0


def test_save_and_load_give_the_same_network(tmp_path):
    """rhd_surrogate_save / rhd_surrogate_load: parameters, standardisation,
    predictions and the warm start of the reloaded network are those of the
    saved one, bit for bit."""
    sur, p, norm = _random_net(16, 99)
    path = str(tmp_path / "net.bin")
    sur.save(path)
    back = rhd.Surrogate.load(path)
    assert (back.n_groups, back.n_features, back.n_outputs, back.n_params) == (
        sur.n_groups, sur.n_features, sur.n_outputs, sur.n_params)
    p1, n1 = sur.get_params()
    p2, n2 = back.get_params()
    assert torch.equal(p1, p2) and torch.equal(n1, n2)
    x = torch.randn(300, sur.n_features, device="cuda")
    assert torch.equal(sur.predict(x), back.predict(x))
    w = synth.preset("mixed_128cube_ng16", n_cells=333, seed=4, device="cuda")
    kw = dict(dt=w.dt, c_v=w.c_v, consts=w.consts)
    e1, r1 = sur.warm_start(w.state, w.edges, w.law, **kw)
    e2, r2 = back.warm_start(w.state, w.edges, w.law, **kw)
    assert torch.equal(e1, e2) and torch.equal(r1, r2)


@pytest.mark.parametrize("G,n", [(4, 256), (32, 1024)])
def test_gradients_match_the_reference_network(G, n):
    sur, p, norm = _random_net(G, 5 + G)
    rng = np.random.default_rng(100 + G)
    x = rng.normal(0, 1.5, (n, sur.n_features)).astype(np.float32)
    y = rng.normal(0, 1.0, (n, sur.n_outputs)).astype(np.float32)
    loss, grad = sur.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
    L, g = M.loss_grad(p, norm, x.astype(np.float64), y.astype(np.float64), sur.n_features,
                       sur.n_outputs, bf=True)
    grad = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - L) < 1e-3 * L
    k = 0
    for l, (o, i) in enumerate(M.shapes(sur.n_features, sur.n_outputs)):
        ew = _rel(grad[k:k + o * i], g[k:k + o * i])
        eb = _rel(grad[k + o * i:k + o * i + o], g[k + o * i:k + o * i + o])
        print(f"G={G} layer {l + 1}: dW rel {ew:.2e}, db rel {eb:.2e}")
        assert ew < 1e-2 and eb < 1e-2, (l, ew, eb)
        k += o * i + o
    assert sur.error_flag() == 0


def _trained(G=16, n_train=1 << 17, seed=7, epochs=4):
    w = synth.preset("mixed_128cube_ng16", n_cells=8, n_groups=G)
    sur = rhd.Surrogate(G, seed)
    x, y = surrogate.training_set(sur, n_train, w.edges, w.law, v_max=1e-2, tau_max=1e4,
                                  seed=seed, device="cuda")
    losses = surrogate.train(sur, x, y, epochs=epochs, batch=4096, seed=seed)
    return sur, w, losses


def test_training_on_solver_data_reduces_the_loss():
    sur, _, losses = _trained(epochs=4)
    print("epoch losses", losses)
    # standardised targets: predicting their mean scores 1
    assert losses[-1] < 0.15 and losses[-1] < 0.5 * losses[0]
    assert sur.error_flag() == 0


def _solve(sur, w, precision, state=None, **kw):
    st = {k: (None if v is None else v.cuda().clone()) for k, v in (state or w.state).items()}
    n = st["rho"].shape[0]
    status = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    iters = torch.zeros(n, dtype=torch.uint8, device="cuda")
    args = dict(dt=w.dt, c_v=w.c_v, consts=w.consts, precision=precision, status=status,
                iters=iters, **kw)
    if sur is None:
        rhd.source_update(st, w.edges, w.law, **args)
    else:
        sur.source_update(st, w.edges, w.law, **args)
    torch.cuda.synchronize()
    out = synth.to_numpy(st)
    out["status"] = status.cpu().numpy().astype(np.int32)
    out["iters"] = iters.cpu().numpy().astype(np.int32)
    return out


def test_warm_started_solve_matches_the_oracle_and_saves_iterations():
    sur, w0, _ = _trained()
    # evaluation cells: same groups and law, other state seed
    st = synth.make_state(1500, w0.edges, w0.law, v_max=1e-2, tau_max=1e4, seed=4242)
    w = synth.Workload("eval", st, w0.edges, w0.law)
    o = run_oracle(w)
    st0 = synth.to_numpy(w.state)
    cold = _solve(None, w, rhd.FP64, **TIGHT)
    warm = _solve(sur, w, rhd.FP64, **TIGHT)
    ok = agreed("fp64 cold and warm-started", cold, warm, oracle=o, fallback_ok=True)
    e = errors(select(warm, ok), select(o, ok), select(st0, ok), w.consts["c"], w.c_v,
               floor=FLOOR)
    print("fp64+surrogate", " ".join(f"{k}={v:.2e}" for k, v in e.items()))
    for k, v in e.items():
        if not k.endswith("_plain"):
            assert v < FP64_TOL, (k, v)
    ce, cm = conservation(select(warm, ok), select(st0, ok), w.consts["c"], w.consts["c_hat"])
    assert ce < 64 * 2.0 ** -52 and cm < 64 * 2.0 ** -52
    fb = float((warm["status"] == rhd.STATUS_FALLBACK).mean())
    print(f"Newton iterations per cell: cold {cold['iters'].mean():.2f}, "
          f"surrogate {warm['iters'].mean():.2f}; fallback fraction {fb:.4f}")
    assert warm["iters"].mean() < cold["iters"].mean()
    assert fb < 0.05
    # mixed form from the surrogate's guess, default tolerances: the stated bound
    mixed = _solve(sur, w, rhd.MIXED)
    okm = agreed("mixed warm-started", mixed, oracle=o, fallback_ok=True)
    em = errors(select(mixed, okm), select(o, okm), select(st0, okm), w.consts["c"], w.c_v, floor=DEFAULT_FLOOR)
    print("mixed+surrogate", " ".join(f"{k}={v:.2e}" for k, v in em.items()))
    assert em["T"] < MIXED_BOUND and em["erad"] < MIXED_BOUND and em["egas"] < MIXED_BOUND


def test_a_useless_surrogate_falls_back_to_the_cold_start():
    """Output bias far off (T x e^5, E_g x e^30) and a Newton cap the cold
    start meets but the bad guess does not: the cells fall back and still
    come out as the oracle gives them."""
    G = 4
    w = synth.preset("tiny", n_cells=600, seed=31)
    sur = rhd.Surrogate(G, 3)
    p, norm = sur.get_params()
    p = p.cpu().numpy()
    nin, nout = sur.n_features, sur.n_outputs
    off = sum(o * i + o for o, i in M.shapes(nin, nout)[:3])
    p[off:off + nout * M.H] = 0.0
    p[off + nout * M.H:] = np.array([5.0] + [30.0] * G, dtype=np.float32)
    sur.set_params(torch.tensor(p, device="cuda"))
    o = run_oracle(w)
    st0 = synth.to_numpy(w.state)
    cap = dict(max_newton=12, **TIGHT)
    cold = _solve(None, w, rhd.FP64, **cap)
    warm = _solve(sur, w, rhd.FP64, **cap)
    n_fb = int((warm["status"] == rhd.STATUS_FALLBACK).sum())
    print("status counts cold", np.bincount(cold["status"], minlength=4), "warm",
          np.bincount(warm["status"], minlength=4))
    assert n_fb > 0.5 * len(warm["status"])
    ok = converged(cold, o) & (warm["status"] <= rhd.STATUS_FALLBACK)
    assert (ok == converged(cold, o)).all()
    e = errors(select(warm, ok), select(o, ok), select(st0, ok), w.consts["c"], w.c_v,
               floor=FLOOR)
    for k, v in e.items():
        if not k.endswith("_plain"):
            assert v < FP64_TOL, (k, v)


def test_a_tensor_core_wait_that_runs_out_is_reported_and_the_device_stays_usable():
    """The bounded waits of the tensor-core GEMM: with the test switch on, no
    MMA is issued, so the first barrier wait gives up after a few polls with
    nothing in flight; the kernel sets the surrogate's error flag, frees its
    tensor memory and returns.  Afterwards the same device trains and
    predicts normally (a fresh surrogate: flag 0, forward as the reference)."""
    G, n = 4, 257
    sur, p, norm = _random_net(G, 5)
    x = torch.tensor(np.random.default_rng(1).normal(0, 1, (n, sur.n_features)).astype(np.float32),
                     device="cuda")
    sur.test_wait_timeout(True)
    sur.predict(x)
    torch.cuda.synchronize()
    assert sur.error_flag() == 1
    sur.test_wait_timeout(False)
    fresh, p2, norm2 = _random_net(G, 6)
    y = fresh.predict(x).cpu().numpy().astype(np.float64)
    ref = M.predict(p2, norm2, x.cpu().numpy().astype(np.float64), fresh.n_features,
                    fresh.n_outputs, bf=True)
    assert _rel(y, ref) < 1e-2
    assert fresh.error_flag() == 0
    # and a training step on the fresh network runs its backward GEMMs cleanly
    yt = torch.tensor(np.random.default_rng(2).normal(0, 1, (n, fresh.n_outputs)).astype(np.float32),
                      device="cuda")
    fresh.fit_normalization(x, yt)
    fresh.train_step(x, yt, 0, 256, 1, 0, 1e-3)  # a batch of 256 rows (a multiple of 8)
    torch.cuda.synchronize()
    assert fresh.error_flag() == 0
