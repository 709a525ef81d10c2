"""QPD sampling and h-TN simplification on the GPU (section 4.3; Step 1 of
section 6.1) against the oracle: the sampled network's tensors element by
element (bit-exact: the fused CT products, the draws and the copies are the
same FP64 operations in the same order), its kept sizes, and the contraction
of the sampled network."""
import numpy as np
import pytest

import synth
from oracle import sampling
from tests.gpu_util import FP64_TOL, REL_TOL, oracle_value, rel_err, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def _handle(net):
    from paper_2410_15080_b300.htn import HTN
    h = HTN(0)
    for inds, data, kind in to_device(net):
        h.add_tensor(inds, data=data, kind=kind)
    h.set_output(net.output)
    return h


def _uniforms(n_groups, s, seed):
    import torch
    u = np.random.default_rng(seed).uniform(0, 1, (max(n_groups, 1), s))
    return u, torch.from_numpy(u.ravel().copy()).cuda()


def _check_against_oracle(net, s, seed):
    import torch
    h = _handle(net)
    ng = h.qpd_groups()
    u, ud = _uniforms(ng, s, seed)
    hs = h.qpd_sample(s, ud)
    torch.cuda.synchronize()
    kinds = [t.kind for t in net.tensors]
    ot, ok, info = sampling.qpd_sample(net.pairs(), kinds, net.output, s, u)
    assert hs.n_tensors == len(ot) and ng == len(info)
    assert hs.qpd_info() == [(d, len(k)) for d, k in info]
    for t, (inds, arr) in enumerate(ot):
        ti = hs.tensor_info(t)
        assert ti["inds"] == tuple(inds) and ti["dims"] == tuple(np.shape(arr)), (t, ti)
        got = hs.tensor_view(t).cpu().numpy()
        assert got.dtype == np.asarray(arr).dtype
        np.testing.assert_array_equal(got, arr)
    return h, hs, ot, info


@pytest.mark.parametrize("s", [1, 7, 100])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sampled_network_equals_the_oracle(s, dtype):
    net = synth.ring_htn(n_sub=4, gates_per_edge=2, wires_per_edge=1, k=3, seed=s, dtype=dtype)
    h, hs, ot, info = _check_against_oracle(net, s, seed=100 + s)
    assert all(1 <= len(k) <= min(s, d) for d, k in info)
    # the contraction of the sampled network
    ref = oracle_value(synth.HTN([synth.Tensor("QT", i, a) for i, a in ot], net.output))
    for prec, tol in (("fp64", FP64_TOL), ("bf16x3", REL_TOL)):
        hp = hs if prec == "fp64" else None
        if hp is None:
            hp = h.qpd_sample(s, _uniforms(h.qpd_groups(), s, 100 + s)[1])
        hp.plan(prec)
        out = hp.contract()
        hp.sync()
        err = rel_err(out.cpu().numpy(), ref)
        assert err <= tol, (prec, err)
        hp.close()
    h.close()


def test_mixed_groups_sizes_and_chords():
    """Ring edges with one gate cut (a group of one CT) and chords with two:
    the groups of the 100-qubit network's topology on a small instance."""
    net = synth.ring_chords_htn(k=2, n_sub=6, n_chords=3, chord_step=2, seed=3)
    h, hs, ot, info = _check_against_oracle(net, 20, seed=5)
    assert sorted({d for d, _ in info}) == [6, 36]
    hs.close()
    h.close()


def test_network_without_gate_groups_is_unchanged():
    """Only wire cuts: nothing is sampled; the new network borrows the same
    tensors and contracts to the same value."""
    net = synth.ring_htn(n_sub=3, gates_per_edge=0, wires_per_edge=2, k=2, seed=2)
    h = _handle(net)
    assert h.qpd_groups() == 0
    hs = h.qpd_sample(10, None)
    assert hs.qpd_info() == [] and hs.n_tensors == len(net.tensors)
    hs.plan("fp64")
    out = hs.contract()
    hs.sync()
    assert rel_err(out.cpu().numpy(), oracle_value(net)) <= FP64_TOL
    hs.close()
    h.close()


def test_unbiased_over_seeds():
    """The mean of the sampled estimate over 200 seeds is within 4 standard
    errors of the exact value (all on the GPU, FP64 path)."""
    import torch
    net = synth.ring_htn(n_sub=3, gates_per_edge=1, wires_per_edge=1, k=1, seed=4)
    exact = oracle_value(net)[0]
    h = _handle(net)
    est = []
    for seed in range(200):
        hs = h.qpd_sample(8, _uniforms(h.qpd_groups(), 8, seed)[1])
        hs.plan("fp64")
        out = hs.contract()
        hs.sync()
        est.append(float(out.cpu()[0]))
        hs.close()
    torch.cuda.synchronize()
    h.close()
    est = np.array(est)
    se = est.std(ddof=1) / np.sqrt(len(est))
    assert abs(est.mean() - exact) <= 4 * se


def test_100_qubit_network_sampled_at_full_size():
    """The 100-qubit network (2 GB of QTs): s = 20 draws per group.  Fused
    CTs, draws and kept values equal the oracle's on the group vectors; the
    truncated QTs are checked entry by entry at 4096 sampled positions each
    against the source QT; the sampled network contracts to the oracle's
    value of the same sampled network on the entries k in {0, 1}."""
    import torch
    from tests.gpu_util import oracle_restricted
    net = synth.ring_chords_htn()
    h = _handle(net)
    ng = h.qpd_groups()
    assert ng == 20  # 12 ring edges (1 gate cut) + 8 chords (2 gate cuts)
    s = 20
    u, ud = _uniforms(ng, s, 77)
    hs = h.qpd_sample(s, ud)
    torch.cuda.synchronize()
    kinds = [t.kind for t in net.tensors]
    groups = sampling.gate_groups(net.pairs(), kinds, net.output)
    n_other = hs.n_tensors - ng
    keep = []
    for x, (a, b, cts, inds) in enumerate(groups):
        c = sampling.fused_ct([net.tensors[t].data for t in cts])
        cnt = sampling.draw_counts(c, s, u[x])
        k = np.nonzero(cnt)[0]
        keep.append(k)
        got = hs.tensor_view(n_other + x).cpu().numpy()
        np.testing.assert_array_equal(got, sampling.sampled_ct(c, cnt, s)[k])
    # truncated QTs: sampled entries against the source (fuse order of the
    # oracle: groups in order, each at the first of its axes)
    rng = np.random.default_rng(1)
    t_new = 0
    max_id = max(i for t in net.tensors for i in t.inds)
    dropped = {t for g in groups for t in g[2]}
    for t, T in enumerate(net.tensors):
        if t in dropped:
            continue
        ti = hs.tensor_info(t_new)
        view = hs.tensor_view(t_new)
        t_new += 1
        if T.kind != "QT":
            continue
        mine = [x for x, g in enumerate(groups) if t in g[:2]]
        if not mine:
            continue
        # axis map of the truncated QT
        axes = [(i, None) for i in T.inds]
        for x in mine:
            pos = [j for j, (i, g) in enumerate(axes) if g is None and i in groups[x][3]]
            first = min(pos)
            nx = []
            for j, a in enumerate(axes):
                if j == first:
                    nx.append((max_id + 1 + x, x))
                if j not in pos:
                    nx.append(a)
            axes = nx
        assert ti["inds"] == tuple(i for i, _ in axes)
        flat = view.reshape(-1)
        idx = rng.integers(0, flat.numel(), 4096)
        got = flat[torch.from_numpy(idx).cuda()].cpu().numpy()
        coords = np.unravel_index(idx, ti["dims"])
        src_idx = {i: None for i in T.inds}
        for (i, g), cvec in zip(axes, coords):
            if g is None:
                src_idx[i] = cvec
            else:
                f = keep[g][cvec]
                dims = [T.data.shape[T.inds.index(j)] for j in groups[g][3]]
                digits = np.unravel_index(f, dims)
                for j, dgt in zip(groups[g][3], digits):
                    src_idx[j] = dgt
        want = T.data[tuple(src_idx[i] for i in T.inds)]
        np.testing.assert_array_equal(got, want)
    # the contraction of the sampled network against the oracle's
    ot, ok, info = sampling.qpd_sample(net.pairs(), kinds, net.output, s, u)
    onet = synth.HTN([synth.Tensor(k_, i, a) for (i, a), k_ in zip(ot, ok)], net.output)
    ref = oracle_restricted(onet)
    hs.plan("bf16x3", max_intermediate_bytes=8 << 30, n_candidates=64)
    out = hs.contract()
    hs.sync()
    got = out.cpu().numpy()[:2]
    assert rel_err(got, ref) <= REL_TOL
    hs.close()
    h.close()
