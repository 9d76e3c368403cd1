"""GPU parity of the troubled-cell indicator: criterion flags, network inputs,
tensor-core inference, and the training gradient, against the FP64 oracle.

Integer decisions (flags) are compared where the oracle's decision is not a near
tie; the rest must still be a valid answer (one of the two).  The network runs on
bfloat16 weights (and bfloat16 activations on the tensor cores) with FP32
accumulation, so logits are compared with a tolerance of a few bfloat16 ulps of the
activations, and gradients (FP32 sums over the batch) to 1e-3 relative.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu

_cache = {}


def case(name):
    if name not in _cache:
        if name == "riemann2d":
            w = synth.workload("euler2d_riemann", size=24, q=2)
        else:
            w = synth.workload("euler3d_tet64", size=6, q=2)
            # add a density jump so the criterion has something to flag
            m = w["mesh"]
            O = oracle.Oracle(m)
            jump = (O.xc[:, 0] > 0.5)
            w["u0"] = w["u0"] * np.where(jump, 1.0, 0.6)[None]
        w["O"] = oracle.Oracle(w["mesh"])
        _cache[name] = w
    return _cache[name]


def dev(M, u):
    return torch.from_numpy(M.to_lib(np.ascontiguousarray(u))).cuda()


@pytest.mark.parametrize("name", ["riemann2d", "tet3d"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_criterion_flags(name, prec):
    w = case(name)
    O = w["O"]
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision=prec, **w["scheme"])
    ws = dg.workspace(M, sch)
    fl = torch.zeros(M.n_cells, dtype=torch.uint8, device="cuda")
    dg.dolinc_criterion(M, sch, dev(M, w["u0"]), fl, ws)
    got = M.from_lib(fl.cpu().numpy())
    want = O.criterion(w["u0"], oracle.Scheme(**w["scheme"]))
    assert want.sum() > 0 and want.sum() < O.n_cells
    agree = (got == want).mean()
    if prec == "fp64":
        assert agree == 1.0, (agree, np.nonzero(got != want))
    else:
        assert agree > 0.995, agree          # decisions near the thresholds taken in FP32


@pytest.mark.parametrize("name", ["riemann2d", "tet3d"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_network_inputs(name, prec):
    """Own features element by element; the three neighbour blocks are the top three of
    the cell's face neighbours in lexicographic order, which is not unique on near-ties
    (piecewise-constant data makes many), so each block must be one of the cell's
    neighbours' feature vectors and the blocks' first keys must sum to the oracle's."""
    w = case(name)
    O = w["O"]
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision=prec, **w["scheme"])
    ws = dg.workspace(M, sch)
    x = torch.zeros((M.n_cells, 24), dtype=torch.float32, device="cuda")
    dg.dolinc_indicator_features(M, sch, dev(M, w["u0"]), x, ws)
    got = x.cpu().numpy()[M.perm]
    own, want = O.features(w["u0"], oracle.Scheme(**w["scheme"]))
    tol = (1e-5 if prec == "fp64" else 3e-4) * (1 + np.abs(want).max())
    np.testing.assert_allclose(got[:, :6], want[:, :6], atol=tol)
    nbrs = [[] for _ in range(O.n_cells)]
    for P, Q in zip(O.owner, O.neigh):
        nbrs[P].append(Q if Q >= 0 else P)
        if Q >= 0:
            nbrs[Q].append(P)
    for c in range(O.n_cells):
        cand = own[nbrs[c]]
        for a in range(3):
            blk = got[c, 6 + 6 * a: 12 + 6 * a]
            assert np.abs(cand - blk).max(axis=1).min() <= tol, (c, a)
        assert abs(got[c, 6::6][:3].sum() - want[c, 6::6][:3].sum()) <= 3 * tol, c


@pytest.mark.parametrize("name", ["riemann2d", "tet3d"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_inference_equals_features_then_network(name, prec):
    """dolinc_indicator_infer without an input buffer gathers each cell's 24 inputs
    inside the network kernel; logits and flags equal the features pass followed by
    the network on the written inputs, bit for bit."""
    w = case(name)
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision=prec, **w["scheme"])
    ws = dg.workspace(M, sch)
    net = dg.MLP(seed=5)
    u = dev(M, w["u0"])
    x = torch.zeros((M.n_cells, 24), dtype=torch.float32, device="cuda")
    out = []
    for buf in (x, None):
        lg = torch.zeros(M.n_cells, dtype=torch.float32, device="cuda")
        fl = torch.zeros(M.n_cells, dtype=torch.uint8, device="cuda")
        dg.dolinc_indicator_infer(M, sch, net, u, buf, fl, ws, logits=lg)
        out.append((lg.cpu().numpy(), fl.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert 0 < out[0][1].sum() < M.n_cells or np.abs(out[0][0]).max() > 0


def test_tensor_core_inference_matches_bf16_reference():
    rng = np.random.default_rng(3)
    theta = omlp.init(7)
    theta[omlp.N_PARAMS - 1] = 0.1
    X = np.abs(rng.normal(size=(1000, 24))).astype(np.float32)
    net = dg.MLP(seed=1)
    net.set_params(theta)
    xd = torch.from_numpy(X).cuda()
    lg = torch.zeros(1000, dtype=torch.float32, device="cuda")
    fl = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    net.forward(xd, lg, fl)
    got = lg.cpu().numpy()
    want, _ = omlp.forward(theta, X, weights_bf16=True, act_bf16=True)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() < 2e-2 * scale
    clear = np.abs(want) > 0.05 * scale
    assert np.all((fl.cpu().numpy()[clear] > 0) == (want[clear] > 0))


@pytest.mark.parametrize("n", [37, 2048])
def test_training_gradient_matches_oracle(n):
    rng = np.random.default_rng(n)
    theta = omlp.init(11)
    X = np.abs(rng.normal(size=(n, 24))).astype(np.float32)
    y = (rng.uniform(size=n) < 0.2).astype(np.uint8)
    net = dg.MLP(seed=2)
    net.set_params(theta)
    g = torch.zeros(dg.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 3.0, g, loss)
    L, G = omlp.loss_and_grad(theta, X.astype(np.float64), y, pos_weight=3.0, weights_bf16=True)
    assert abs(loss.item() - L) < 1e-4 * abs(L)
    gg = g.cpu().numpy()
    assert np.abs(gg - G).max() < 1e-3 * np.abs(G).max()


def test_training_reduces_loss():
    rng = np.random.default_rng(5)
    n = 8192
    X = np.abs(rng.normal(size=(n, 24))).astype(np.float32)
    y = ((X[:, 0] + 0.5 * X[:, 7] - X[:, 13]) > 0.6).astype(np.uint8)
    net = dg.MLP(seed=3)
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(xd, yd, 1.0, None, loss)
    l0 = loss.item()
    for _ in range(300):
        net.train_step(xd, yd, 3e-3, 1.0, loss)
    net.loss_grad(xd, yd, 1.0, None, loss)
    assert loss.item() < 0.3 * l0
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    net.forward(xd, None, fl)
    acc = (fl.cpu().numpy() == y).mean()
    assert acc > 0.95, acc


def test_trained_network_keeps_a_riemann_run_finite():
    """What the learned indicator gains over the method without it: trained on the
    criterion's labels of four seeded Riemann runs, the network switches the
    first-order fallback on a held-out problem whose unlimited run breaks down at
    once; the network-switched run stays finite with positive density and lands
    close to the criterion-switched run, and it flags nearly every cell the criterion
    flags."""
    from paper_2404_08952_gb300 import indicator as ind
    mk = lambda sd: synth.workload("euler2d_riemann", size=48, order=sd, q=2)
    Xs, Ys = [], []
    for x, y in ind.riemann_runs(mk, range(4), 30, 2, precision="fp32"):
        Xs.append(x)
        Ys.append(y)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    net = dg.MLP(seed=4)
    hist, _ = ind.train(net, X, Y, epochs=25, batch=4096, lr=2e-3)
    assert hist[-1] < hist[0]
    w = mk(1000)
    steps = 40
    st_none, fin_none, _, _ = ind.run_with(w, "none", steps, precision="fp32")
    st_crit, fin_crit, _, fl_crit = ind.run_with(w, "criterion", steps, precision="fp32")
    st_net, fin_net, _, fl_net = ind.run_with(w, "network", steps, precision="fp32", net=net)
    assert not fin_none
    assert fin_crit and fin_net
    assert st_net[0].min() > 0
    assert np.abs(st_net - st_crit).sum() / np.abs(st_crit).sum() < 1e-2
    # held-out agreement of the network's flags with the criterion's
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision="fp32", **w["scheme"])
    ws = dg.workspace(M, sch)
    u = torch.from_numpy(M.to_lib(st_crit)).cuda()
    fc = torch.zeros(M.n_cells, dtype=torch.uint8, device="cuda")
    dg.dolinc_criterion(M, sch, u, fc, ws)
    xf = torch.zeros((M.n_cells, 24), dtype=torch.float32, device="cuda")
    dg.dolinc_indicator_features(M, sch, u, xf, ws)
    fn = torch.zeros_like(fc)
    net.forward(xf, None, fn)
    a, b = fn.cpu().numpy() > 0, fc.cpu().numpy() > 0
    # trained with the positive class up-weighted: it flags generously (high recall)
    assert (a == b).mean() > 0.8
    assert (a & b).sum() > 0.85 * b.sum()
