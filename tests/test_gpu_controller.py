"""The learned sweep-type controller: its network kernels against a numpy
reference, the self-generated decision log (state saved and restored between
trial actions) against a replay of the logged actions, and the controlled run
against the eps rule of Algorithm 3."""
import numpy as np
import pytest
import torch

from paper_1811_10573_gb300 import controller, cpals, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1811_10573_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def np_forward(params, X):
    F, H = cpals.CTRL_FEATURES, 32
    W1 = params[:H * F].reshape(H, F).astype(np.float64)
    b1 = params[H * F:H * F + H]
    W2 = params[H * F + H:H * F + H + 3 * H].reshape(3, H)
    b2 = params[H * F + H + 3 * H:]
    h = np.maximum(X @ W1.T + b1, 0)
    z = h @ W2.T + b2
    z -= z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def np_loss(params, X, y, w):
    p = np_forward(params, X)
    return float(-np.sum(w * np.log(p[np.arange(len(y)), y])) / np.sum(w))


def test_mlp_forward_matches_numpy():
    rng = np.random.default_rng(0)
    params = controller.init_params(3) + 0.05 * rng.standard_normal(cpals.CTRL_PARAMS).astype(np.float32)
    X = rng.standard_normal((257, cpals.CTRL_FEATURES)).astype(np.float32)
    got = cpals.mlp_forward(params, X)
    assert np.max(np.abs(got - np_forward(params.astype(np.float64), X.astype(np.float64)))) < 1e-5


def test_mlp_training_step_follows_the_gradient_and_fits():
    """One Adam step moves every parameter with a clear gradient against it
    (numpy central differences); many steps fit a separable labelling."""
    rng = np.random.default_rng(1)
    n = 300
    X = rng.standard_normal((n, cpals.CTRL_FEATURES)).astype(np.float32)
    y = (np.argmax(X[:, :3] + 0.5 * X[:, 3:6], axis=1)).astype(np.int32)
    w = controller.class_weights(y)
    p0 = controller.init_params(2)
    p1, _ = cpals.mlp_train(X, y, w, p0, epochs=1, lr=1e-3, decay=0.0)
    step = (p1 - p0).astype(np.float64)
    h = 1e-3
    checked = 0
    for q in rng.choice(cpals.CTRL_PARAMS, 60, replace=False):
        e = np.zeros(cpals.CTRL_PARAMS)
        e[q] = h
        g = (np_loss(p0 + e, X, y, w) - np_loss(p0 - e, X, y, w)) / (2 * h)
        if abs(g) > 1e-3:
            assert np.sign(step[q]) == -np.sign(g), (q, g, step[q])
            checked += 1
    assert checked >= 10
    p, loss = cpals.mlp_train(X, y, w, p0, epochs=1500, lr=1e-2, decay=0.0)
    pred = np.argmax(cpals.mlp_forward(p, X), axis=1)
    assert loss < 0.2 and np.mean(pred == y) > 0.95


def _problem():
    return synth.make_problem("collinear", [48, 44, 40], 12, seed=4, noise=1e-2, collinearity=0.8,
                              init="uniform", storage="f32", eps=0.1, sweeps=60)


def _ctx(p, prec):
    g = cpals.CPALS(p.dims, p.R, prec)
    g.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    g.init_factors(p.A0)
    return g


@pytest.mark.parametrize("to_target", [False, True], ids=["gain_rate", "time_to_target"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_controller_log_restores_state_between_trials(prec, to_target):
    """After the log, the context holds exactly the state reached by applying
    the logged actions one after the other from the start: every trial was
    undone (factors compared bit for bit), with either label rule (trials to
    a target fitness run Algorithm 3 after the candidate, operator rebuilds
    included, and the log ends where the trajectory reaches the target)."""
    p = _problem()
    with _ctx(p, prec) as g:
        if to_target:
            f_als = float(g.run(40, 0.0, True, 0.0)["fitness"][-1])
            g.init_factors(p.A0)
            g.set_pp_stop_tol(1e-6)
            g.set_controller_labels(f_als - 1e-6, 40)
        log = g.controller_log(40, 0.1, True)
        A_log = g.get_factors()
    labels = log["labels"]
    assert 0 < len(labels) <= 40 if to_target else len(labels) == 40
    assert set(np.unique(labels)) <= {0, 1, 2}
    for t, lab in enumerate(labels):
        assert np.isfinite(log["gains"][t, lab]) and log["costs"][t, lab] > 0
    with _ctx(p, prec) as g:
        for lab in labels:
            if lab == 1:
                g.als_sweep()
            elif lab == 2:
                g.pp_build_operators()
                g.pp_sweep(True)
            else:
                g.pp_sweep(True)
        A_rep = g.get_factors()
    for a, b in zip(A_log, A_rep):
        np.testing.assert_array_equal(a, b)


def test_run_controlled_without_network_is_the_eps_rule():
    p = _problem()
    with _ctx(p, "fp64") as g:
        ref = g.run(50, 0.1, True, 0.0)
    with _ctx(p, "fp64") as g:
        out = g.run_controlled(50, 0.1, True, 0.0)
    assert out["kinds"] == ref["kinds"]
    assert not np.any(out["learned"])
    np.testing.assert_allclose(out["fitness"], ref["fitness"], rtol=0, atol=1e-12)


def test_run_controlled_network_decides():
    """A network whose output bias always names the ALS sweep drives a run
    identical to plain ALS, every decision taken by the network."""
    p = _problem()
    params = np.zeros(cpals.CTRL_PARAMS, dtype=np.float32)
    params[-3:] = [0.0, 10.0, 0.0]                     # b2: ALS
    with _ctx(p, "fp64") as g:
        ref = g.run(30, 0.0, True, 0.0)                # eps = 0: ALS only
    with _ctx(p, "fp64") as g:
        g.set_controller(params, 0.6)
        out = g.run_controlled(30, 0.1, True, 0.0)
    assert out["kinds"] == ["als"] * 30 and np.all(out["learned"])
    np.testing.assert_array_equal(out["fitness"], ref["fitness"])


def _forced(action):
    """A network whose output bias always names one action (0 PP, 1 ALS,
    2 rebuild + PP) with probability ~1."""
    params = np.zeros(cpals.CTRL_PARAMS, dtype=np.float32)
    b2 = [0.0, 0.0, 0.0]
    b2[action] = 10.0
    params[-3:] = b2
    return params


@pytest.mark.parametrize("net", ["always_als", "always_rebuild", "trained"])
@pytest.mark.parametrize("tol", [0.0, 1e-5])
def test_controlled_run_device_loop_equals_host_loop(net, tol):
    """cpals_run_controlled with its decisions in the device loop (history,
    features and forward pass in the decide kernel) against the host loop:
    the same sweep kinds, the same learned/rule source of every decision and
    bit-identical fitness traces and factors, for networks that always name
    one action (ALS; operator rebuild + PP sweep) and for the committed
    network, which decides by its features."""
    p = _problem()
    params = {"always_als": _forced(1), "always_rebuild": _forced(2)}.get(net)
    if params is None:
        params = controller.load()
        if params is None:
            pytest.skip("no committed controller parameters")
    outs, facs = [], []
    for loop in (True, False):
        with _ctx(p, "fp64") as g:
            g.set_pp_stop_tol(tol)
            g.set_device_loop(loop)
            g.set_controller(params, 0.6)
            outs.append(g.run_controlled(60, 0.1, True, 0.0))
            facs.append(g.get_factors())
    dev, host = outs
    assert dev["kinds"] == host["kinds"]
    assert np.array_equal(dev["learned"], host["learned"])
    assert np.array_equal(dev["fitness"], host["fitness"])
    for a, b in zip(*facs):
        assert np.array_equal(a, b)
    if net == "always_als":
        assert dev["kinds"] == ["als"] * 60 and np.all(dev["learned"])
    if net == "always_rebuild":
        assert dev["kinds"] == ["pp_init"] * 60 and np.all(dev["learned"])
