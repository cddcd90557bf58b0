"""Learned warm start and block preconditioner on the GPU.

Against the oracle network (same bfloat16-rounded weights): the network
inputs built from the assembled system, the forward pass, P and x0, the
energy-norm loss, every gradient tensor, the training pair and one Adam step.
Then the solver with the learned parts (the FP64 residual still decides
convergence) and what training gains on held-out steps of a loaf.

Tolerances: the GPU network runs FP32 activations and accumulations on the
same bfloat16 weights as the oracle, so outputs, loss and gradients agree to
about K u (K <= 128 terms per sum, u = 6e-8 for FP32): 1e-5 relative, taken
norm-wise per tensor; inputs are O(1) and agree to 1e-5 absolute.
"""
import numpy as np
import pytest

from helpers import RTOL64, deformed_state, gpu_material, oracle_model
from oracle import gnn as og
from workloads import beam_config, he_normal_weights, loaf_config, LOAF_AXES

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2103_14870_gb300 as gf  # noqa: E402

RTOL_NET = 1e-5
ABS_IN = 1e-5
SHAPES = list(og.param_shapes().items())


def active_weights(seed):
    """He-normal weights with a small non-zero decoder and small random biases,
    so that every path of the network carries gradient."""
    w = he_normal_weights(SHAPES, seed=seed, scale={"Wd": 0.05})
    rng = np.random.default_rng(seed + 100)
    o = 0
    for _, shp in SHAPES:
        n = int(np.prod(shp))
        if len(shp) == 1:
            w[o:o + n] = 0.05 * rng.normal(size=n)
        o += n
    return w


def rel_max(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def two_beam_steps():
    """GPU and oracle: two steps of the beam from the same deformed state."""
    w = beam_config()
    model = oracle_model(w)
    m = gf.mesh_create(w.nodes, w.tets, gpu_material(gf, w), cg_rtol=1e-13, cg_maxit=20000)
    st = deformed_state(w, seed=1)
    m.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
    m.step(w.dt, w.f_ext.ravel(), w.pinned)
    st1, info1 = model.step(st, w.dt, w.f_ext, w.pinned)
    return w, model, m, st1, info1


@pytest.mark.parametrize("kernels", [gf.GNN_TENSOR_CORES, gf.GNN_FP32_FMA], ids=["tcgen05", "fp32_fma"])
def test_network_forward_loss_gradients_and_adam_match_oracle(kernels):
    w, model, m, st1, info1 = two_beam_steps()
    wts = active_weights(5)
    params = og.unflatten(og.to_bf16(wts))
    net = gf.Gnn(m, wts)
    net.kernels_set(kernels)
    m.step(w.dt, w.f_ext.ravel(), w.pinned)
    _, info2 = model.step(st1, w.dt, w.f_ext, w.pinned)
    A = info2["A"]
    n = model.n_nodes
    pin = np.zeros(n, bool)
    pin[w.pinned] = True
    bn, tg = og.training_pair(A, info2["b"].reshape(-1, 3), info2["dv"], info1["dv"], pin)

    # the training pair the GPU builds from its own last step (FP64 path):
    # b_net = b - A w cancels, so the floor is 1e-9 of the operands' scale
    b_gpu, t_gpu = net.pair_get()
    scale_b = np.abs(info2["b"]).max() + np.abs(A @ np.where(pin[:, None], info2["dv"], info1["dv"]).ravel()).max()
    assert np.abs(b_gpu - bn.ravel()).max() <= RTOL64 * scale_b
    scale_t = np.abs(info2["dv"]).max() + np.abs(info1["dv"]).max()
    assert np.abs(t_gpu - tg.ravel()).max() <= RTOL64 * scale_t

    g, f, C, s, free, _ = og.build_inputs(A, model.mass, w.nodes, model.edges, pin, bn)
    out_o = og.forward(params, g, f)
    P_o, x0_o, _, _ = og.apply_outputs(out_o, C, bn, s)
    fw = net.forward(bn.ravel())
    assert np.abs(fw["node_in"] - f).max() <= ABS_IN
    assert np.abs(fw["edge_in"] - g.efeat).max() <= ABS_IN
    assert rel_max(fw["out"], out_o) <= RTOL_NET
    assert rel_max(fw["P"], P_o) <= RTOL_NET
    assert rel_max(fw["x0"], x0_o) <= RTOL_NET

    loss_o, grads_o = og.loss_and_grad(params, g, f, C, bn, tg, free, s, A)
    loss_g, grad_g = net.loss_grad(bn.ravel(), tg.ravel())
    assert abs(loss_g - loss_o) <= RTOL_NET * loss_o
    go = og.flatten(grads_o)
    offs = np.cumsum([0] + [int(np.prod(v)) for _, v in SHAPES])
    for i, (name, _) in enumerate(SHAPES):
        a, b = grad_g[offs[i]:offs[i + 1]], go[offs[i]:offs[i + 1]]
        assert np.linalg.norm(a - b) <= RTOL_NET * np.linalg.norm(b), name

    # one Adam step from fresh moments moves each weight by lr g / (|g| + 1e-8)
    lr = 1e-3
    first, _ = net.train(iters=1, lr=lr)
    assert abs(first - loss_o) <= RTOL_NET * loss_o
    moved = net.params_get().astype(np.float64) - wts.astype(np.float64)
    want = -lr * grad_g / (np.abs(grad_g) + 1e-8)
    big = np.abs(grad_g) > 1e-4 * np.abs(grad_g).max()
    np.testing.assert_allclose(moved[big], want[big], rtol=1e-3, atol=1e-9)


def test_tensor_core_and_fp32_kernels_agree_on_a_loaf():
    """The tcgen05 dense layers and edge messages against the FP32 FMA kernels
    on a half-size loaf (13,892 nodes: 109 node tiles with a ragged last one,
    about 1,600 edge tiles): the same FP32-accurate results up to rounding
    order (1e-5 norm-wise per output and per gradient tensor), and not
    bit-identical, which shows that the tensor-core path ran."""
    w = loaf_config(axes=tuple(0.5 * a for a in LOAF_AXES))
    m = gf.mesh_create(w.nodes, w.tets, gf.material(w.young, w.poisson, w.density, threshold=w.threshold,
                                                    radius=w.radius), cg_rtol=1e-6)
    m.step(w.dt, w.f_ext.ravel())
    m.step(w.dt, w.f_ext.ravel())
    net = gf.Gnn(m, active_weights(7))
    b, t = net.pair_get()
    res = {}
    for k in (gf.GNN_TENSOR_CORES, gf.GNN_FP32_FMA):
        net.kernels_set(k)
        fw = net.forward(b)
        res[k] = (fw, *net.loss_grad(b, t))
    (fa, la, ga), (fb, lb, gb) = res[gf.GNN_TENSOR_CORES], res[gf.GNN_FP32_FMA]
    for key in ("out", "P", "x0"):
        assert np.linalg.norm(fa[key] - fb[key]) <= RTOL_NET * np.linalg.norm(fb[key]), key
    assert not np.array_equal(fa["out"], fb["out"])
    assert abs(la - lb) <= RTOL_NET * abs(lb)
    offs = np.cumsum([0] + [int(np.prod(v)) for _, v in SHAPES])
    for i, (name, _) in enumerate(SHAPES):
        a_, b_ = ga[offs[i]:offs[i + 1]], gb[offs[i]:offs[i + 1]]
        assert np.linalg.norm(a_ - b_) <= RTOL_NET * np.linalg.norm(b_), name


def test_zero_decoder_gives_scaled_block_jacobi():
    w, model, m, st1, info1 = two_beam_steps()
    net = gf.Gnn(m, he_normal_weights(SHAPES, seed=2, zero=("Wd",)))
    rng = np.random.default_rng(3)
    b = rng.normal(size=3 * model.n_nodes)
    fw = net.forward(b)
    assert np.abs(fw["out"]).max() == 0.0
    pin = np.zeros(model.n_nodes, bool)
    pin[w.pinned] = True
    *_, Dinv = og.build_inputs(info1["A"], model.mass, w.nodes, model.edges, pin, b.reshape(-1, 3))
    assert rel_max(fw["P"], (1 + og.EPS) * Dinv) <= RTOL_NET
    assert rel_max(fw["x0"], np.einsum("nab,nb->na", (1 + og.EPS) * Dinv, b.reshape(-1, 3))) <= RTOL_NET


@pytest.mark.parametrize("flags", [gf.GNN_START, gf.GNN_PRECOND, gf.GNN_START | gf.GNN_PRECOND])
def test_learned_solve_keeps_the_fp64_residual_and_solution(flags):
    """With learned start and/or blocks, PCG still stops on the FP64 residual
    and lands on the plain solve's solution."""
    w = beam_config()
    mat = gpu_material(gf, w, threshold=np.inf)
    mp = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=1e-10, cg_maxit=20000)
    ml = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=1e-10, cg_maxit=20000)
    net = gf.Gnn(ml, he_normal_weights(SHAPES, seed=4, scale={"Wd": 0.02}))
    st = deformed_state(w, seed=2)
    for mm in (mp, ml):
        mm.state_set(x=st.x.ravel(), v=st.v.ravel(), labels=st.labels, chi=st.chi)
        mm.step(w.dt, w.f_ext.ravel(), w.pinned)
    net.attach(flags)
    for _ in range(3):
        v0 = mp.velocities_get()
        sp_ = mp.step(w.dt, w.f_ext.ravel(), w.pinned)
        sl_ = ml.step(w.dt, w.f_ext.ravel(), w.pinned)
        assert sp_["status"] == 0 and sl_["status"] == 0
        assert sl_["rel_res"] <= 1e-10
        dv = mp.velocities_get() - v0
        assert np.linalg.norm(ml.velocities_get() - mp.velocities_get()) <= 1e-7 * np.linalg.norm(dv)


def test_training_gains_on_held_out_loaf_steps():
    """Online training on 40 steps of a loaf (half-size axes), evaluation on
    the next 10: the trained network's energy-norm error is well below the
    untrained (zero-decoder) network's on the held-out pairs, and the solve
    started from it needs fewer PCG iterations than plain PCG, at the same
    FP64 residual tolerance."""
    w = loaf_config(axes=tuple(0.5 * a for a in LOAF_AXES))
    mat = gf.material(w.young, w.poisson, w.density, threshold=w.threshold, radius=w.radius)
    m = gf.mesh_create(w.nodes, w.tets, mat, cg_rtol=1e-6, cg_maxit=20000)
    init = he_normal_weights(SHAPES, seed=1, zero=("Wd",))
    net = gf.Gnn(m, init)
    f = w.f_ext.ravel()
    for k in range(40):
        m.step(w.dt, f)
        if k:
            net.train(iters=5, lr=1e-5)
    trained = net.params_get()
    x, v = m.positions_get(), m.velocities_get()
    _, lab = m.damage_get()
    chi = m.chi_get()
    # learned start on the held-out steps
    net.attach(gf.GNN_START)
    learned = [m.step(w.dt, f) for _ in range(10)]
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-6 for s in learned)
    # plain PCG on the same steps; losses of both networks on their pairs
    net.attach(0)
    m.state_set(x=x, v=v, labels=lab, chi=chi)
    plain, loss_t, loss_u = [], [], []
    for k in range(10):
        plain.append(m.step(w.dt, f))
        if k == 0:
            continue        # its x_prev is the learned run's last step
        b, t = net.pair_get()
        net.params_set(trained)
        loss_t.append(net.loss_grad(b, t)[0])
        net.params_set(init)
        loss_u.append(net.loss_grad(b, t)[0])
    it_l = np.mean([s["cg_iters"] for s in learned])
    it_p = np.mean([s["cg_iters"] for s in plain])
    assert it_l < it_p, (it_l, it_p)
    assert np.mean(loss_t) < 0.5 * np.mean(loss_u), (np.mean(loss_t), np.mean(loss_u))
