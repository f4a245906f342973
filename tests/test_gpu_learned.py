"""The learned proposal on the GPU: training kernels against the FP64
reference (gradients), Adam against its closed form, cluster labels against
the oracle's pair classes, and the learned boolean query, whose answers must
equal the plain query's exactly whatever the network proposes."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import mlp as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rsi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2305_01867_gb300 as m
    return m


@pytest.fixture(scope="module")
def c1(rsi):
    mesh = W.config_mesh("c1")
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
    info = bvh.info()
    return mesh, bvh, np.array(info["extent_lo"]), np.array(info["extent_hi"])


def _labels_np(lab):
    """[n, 8] int32 bit masks -> [n, 256] float multi-hot."""
    u = lab.astype(np.int64) & 0xFFFFFFFF
    bits = (u[:, :, None] >> np.arange(32)[None, None, :]) & 1
    return bits.reshape(len(lab), 256).astype(np.float64)


def _pack_labels(y):
    """[n, 256] 0/1 -> [n, 8] int32 bit masks (bit c of word c / 32)."""
    b = y.reshape(len(y), 8, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)[None, None, :]
    return b.sum(2).astype(np.uint32).view(np.int32)


def test_cluster_labels_match_oracle(rsi, c1):
    mesh, bvh, _, _ = c1
    F, E = W.rays(W.config_rays("c1", 300), mesh)
    lab = rsi.cluster_labels(bvh, torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()).cpu().numpy()
    cls = oracle.pair_classes(mesh.vertices, mesh.triangles, F, E)
    perm = bvh.export()["perm"]
    leaf_of = np.empty(len(perm), np.int64)
    leaf_of[perm] = np.arange(len(perm))            # triangle -> leaf
    clus = (leaf_of * 256) // len(perm)
    got = _labels_np(lab)
    checked = 0
    for i in range(len(F)):
        if np.any(cls[i] == oracle.PAIR_AMBIGUOUS):
            continue
        want = np.zeros(256)
        want[np.unique(clus[cls[i] == oracle.PAIR_HIT])] = 1
        assert np.array_equal(got[i], want), i
        checked += 1
    assert checked > 250


def test_gradients_match_reference(rsi, c1):
    mesh, bvh, lo, hi = c1
    F, E = W.rays(W.config_rays("c1", 777), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    y = (np.random.default_rng(8).uniform(size=(len(F), 256)) < 0.03).astype(np.float64)
    lab = torch.from_numpy(_pack_labels(y)).cuda()
    params = ref.init_params(11)
    rng = np.random.default_rng(4)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.1, params[k].shape).astype(np.float32).astype(np.float64)
    net = rsi.MLP(1)
    net.set_params(params)
    loss = net.train_step(bvh, dF, dE, lab, apply=False, want_loss=True)
    _, g_gpu = net.get_params(grads=True)
    x = ref.features(F, E, lo, hi)
    logits, cache = ref.forward(params, x)
    assert abs(loss - ref.bce_loss(logits, y)) < 1e-4 * max(1.0, abs(loss))
    g_ref = ref.backward(params, cache, logits, y)
    mag = _magnitude_backward(cache, logits, y)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, b, m = g_gpu[k], g_ref[k], mag[k]
        if k == "W1":
            a, b, m = a[:6], b[:6], m[:6]
        # Element by element.  Every term of a gradient sum has the same
        # operands on both sides except (i) a BF16 rounding of a layer input
        # that lands on the other side of a rounding boundary (one BF16 ulp,
        # at most 2^-8 relative, in a small share of the terms), (ii) logit
        # differences reaching dL/dz3 through the sigmoid (slope <= 1/4) and
        # (iii) FP32 instead of FP64 accumulation.  So the difference is a
        # small fraction of m, the same sum taken over magnitudes.  2^-11 of
        # m has >= 16x room over what this input shows (3e-5 m at most),
        # while |g| itself is typically 3e-3 m (W1) to 0.9 m (b3): a wrong,
        # missing or misplaced element does not fit inside it.
        bound = 2.0 ** -11 * m + 1e-12
        bad = np.abs(a - b) > bound
        assert not bad.any(), (k, int(bad.sum()), float((np.abs(a - b) / np.maximum(m, 1e-30)).max()))
    assert np.all(g_gpu["W1"][6:] == 0.0)   # padded inputs carry no gradient


def _magnitude_backward(cache, logits, y):
    """The reference backward with every factor replaced by its magnitude:
    for each gradient element, the sum of |terms| its FP64 value is the
    signed sum of (the scale against which rounding differences are
    measured)."""
    n = logits.shape[0]
    dz3 = np.abs(1.0 / (1.0 + np.exp(-logits)) - y) / (n * ref.D_OUT)
    m = {"W3": np.abs(cache["a2"]).T @ dz3, "b3": dz3.sum(0)}
    dz2 = (dz3 @ np.abs(cache["W3"]).T) * np.abs(ref.gelu_grad(cache["z2"]))
    m["W2"], m["b2"] = np.abs(cache["a1"]).T @ dz2, dz2.sum(0)
    dz1 = (dz2 @ np.abs(cache["W2"]).T) * np.abs(ref.gelu_grad(cache["z1"]))
    m["W1"], m["b1"] = np.abs(cache["a0"]).T @ dz1, dz1.sum(0)
    return m


def test_adam_step_closed_form(rsi, c1):
    """From zero moments the first Adam step is -lr g / (|g| + eps)."""
    mesh, bvh, _, _ = c1
    F, E = W.rays(W.config_rays("c1", 2048), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    lab = rsi.cluster_labels(bvh, dF, dE)
    net = rsi.MLP(2)
    p0 = net.get_params()
    net.reset_optimizer()
    net.train_step(bvh, dF, dE, lab, lr=1e-2, apply=True)
    p1, g = net.get_params(grads=True)
    for k in p0:
        step = p1[k] - p0[k]
        want = -1e-2 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(step, want, rtol=1e-4, atol=1e-7), k


@pytest.fixture(scope="module")
def trained(rsi, c1):
    """A network trained briefly on 2e5 labelled segments of the c1 kind."""
    mesh, bvh, _, _ = c1
    F, E = W.rays(W.RaySpec("uniform_box", 200_000, seed=11), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    lab = rsi.cluster_labels(bvh, dF, dE)
    net = rsi.MLP(3)
    losses = net.fit(bvh, dF, dE, lab, epochs=4, batch=4096, lr=2e-3)
    return net, losses


def test_training_reduces_loss(rsi, trained):
    net, losses = trained
    assert losses[-1] < 0.5 * losses[0], losses


@pytest.mark.parametrize("n", [1, 127, 129, 50_000])
def test_learned_query_equals_plain(rsi, c1, trained, n):
    mesh, bvh, _, _ = c1
    F, E = W.rays(W.RaySpec("uniform_box", n, seed=12), mesh)
    if n > 100:
        F[7] = np.nan   # undefined segment: ambiguous, hit 0 on both paths
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    plain = bvh.query(dF, dE, "any_hit")
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E) if n >= 50_000 else None
    for net in (trained[0], rsi.MLP(99)):   # trained and untrained proposals
        got = rsi.query_learned(bvh, net, dF, dE, stats=True)
        assert torch.equal(got["hit"], plain["hit"]) and torch.equal(got["ambiguous"], plain["ambiguous"])
        st = got["stats"]
        assert st["proposal_confirmed"] + st["fallback_rays"] == n and st["device_error"] == 0
        if ref is not None:   # and the definition's answers (Sec. 1, boolean mode), not only the plain path's
            h, a = got["hit"].cpu().numpy(), got["ambiguous"].cpu().numpy()
            assert np.array_equal(a, ref["amb_hit"])
            assert np.array_equal(h[a == 0], ref["hit"][a == 0])


def test_trained_proposal_gains(rsi, c1, trained):
    """What the trained network buys against the method without it: the
    tree search it avoids (node fetches of the plain query vs those of the
    learned query's fallback), and against an untrained network the share
    of hits it settles without a tree search."""
    mesh, bvh, _, _ = c1
    F, E = W.rays(W.RaySpec("uniform_box", 100_000, seed=13), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    plain = bvh.query(dF, dE, "any_hit", stats=True)
    hits = int(plain["hit"].sum())
    good = rsi.query_learned(bvh, trained[0], dF, dE, stats=True)["stats"]
    rand = rsi.query_learned(bvh, rsi.MLP(98), dF, dE, stats=True)["stats"]
    # a short training run (about 200 steps) already settles several times
    # more hits without a tree search than an untrained network does ...
    assert good["proposal_confirmed"] > 0.2 * hits, (good, hits)
    assert good["proposal_confirmed"] > 5 * rand["proposal_confirmed"], (good, rand)
    # ... and every settled segment is a tree search not made
    assert good["node_visits"] < 0.9 * plain["stats"]["node_visits"], (good, plain["stats"])
    assert good["node_visits"] < rand["node_visits"]


def test_attached_network_answers_rsi_query(rsi, c1, trained):
    """rsi_mlp_attach: boolean rsi_query calls on the hierarchy go through
    the learned proposal (its counters show it) with the plain answers;
    detaching, or freeing the network, brings back the plain query."""
    mesh, _, _, _ = c1
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
    F, E = W.rays(W.RaySpec("uniform_box", 30_000, seed=14), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    plain = bvh.query(dF, dE, "any_hit", stats=True)
    assert plain["stats"]["proposal_confirmed"] == 0
    bvh.attach(trained[0])
    got = bvh.query(dF, dE, "any_hit", stats=True)
    assert torch.equal(got["hit"], plain["hit"]) and torch.equal(got["ambiguous"], plain["ambiguous"])
    assert got["stats"]["proposal_confirmed"] > 0
    cnt = bvh.query(dF, dE, "count", stats=True)          # other modes: unaffected
    assert cnt["stats"]["proposal_confirmed"] == 0
    bvh.attach(None)
    again = bvh.query(dF, dE, "any_hit", stats=True)
    assert again["stats"]["proposal_confirmed"] == 0 and torch.equal(again["hit"], plain["hit"])
    temp = rsi.MLP(5)
    bvh.attach(temp)
    bvh._net = None          # the binding's reference dropped: freeing the network detaches it
    temp.close()
    after = bvh.query(dF, dE, "any_hit", stats=True)
    assert after["stats"]["proposal_confirmed"] == 0 and torch.equal(after["hit"], plain["hit"])
    bvh.close()
