"""The cost model's perceptron on the GPU (the library's own forward,
backward and Adam kernels) against the FP64 reference with the same
BF16-rounded weights, and the ranking pipeline end to end."""
import numpy as np
import pytest

from oracle import mlp as ref
from tests.gpu_util import REL_TOL, oracle_value, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


@pytest.mark.parametrize("din,hid,B", [(32, 256, 64), (7, 40, 33)])
def test_forward_and_gradients_match_fp64_reference(din, hid, B):
    import torch
    from paper_2410_15080_b300.htn import MLP
    m = MLP(din, hid, seed=3)
    p = m.params()
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (B, din)).astype(np.float32)
    t = rng.normal(0, 1, B).astype(np.float32)
    xg, tg = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = m.forward(xg).cpu().numpy()
    y_ref, _ = ref.forward(p, x, din, hid)
    assert rel_err(y, y_ref) <= 1e-5
    g, loss = m.gradients(xg, tg)
    g_ref = ref.gradients(p, x, t, din, hid)
    assert abs(loss - ref.loss(p, x, t, din, hid)) <= 1e-5 * max(1.0, abs(loss))
    assert rel_err(g, g_ref) <= 1e-3
    m.close()


def test_adam_training_reduces_the_loss():
    import torch
    from paper_2410_15080_b300.htn import MLP
    rng = np.random.default_rng(2)
    x = rng.normal(0, 1, (512, 8)).astype(np.float32)
    t = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2]).astype(np.float32)
    xg, tg = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    m = MLP(8, 64, seed=4)
    first = m.train_step(xg, tg, 3e-3)
    for _ in range(300):
        last = m.train_step(xg, tg, 3e-3)
    assert last < 0.2 * first
    m.close()


def test_cost_model_pipeline_picks_a_plan_that_contracts_exactly():
    """Train on measured candidate plans of a few networks, choose for a new
    one: the chosen plan's result equals the oracle (the model only chooses)."""
    from paper_2410_15080_b300 import costmodel as cm
    X, y, groups, flops = cm.gen_dataset(cm.train_networks(3), per_net=8)
    assert np.isfinite(y).all()
    model = cm.CostModel(hidden=64)
    losses = model.train(X, y, epochs=40, batch=8)
    assert losses[-1] < losses[0]
    net = cm.eval_networks(1)[0]
    f = cm.select_factor(model.predict(X), y, flops, groups)
    cands, im, ie, pred = cm.choose(model, net, f)
    assert len(cands) == 64 and np.isfinite(pred).all()
    _, out = cm.measure(cm.to_device(net), net.output, cands[im][0], reps=1)
    assert rel_err(out.cpu().numpy(), oracle_value(net)) <= REL_TOL
