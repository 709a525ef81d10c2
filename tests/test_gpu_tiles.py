"""GEMM tiles on the GPU: every orientation and N tile of the tensor-core GEMM
(forced through a tile table) against FP64 numpy matmul, in the three
tensor-core precisions; and the tile autotuner (qtpu_htn_autotune) writing
a table that a later plan follows, with the result still matching the
oracle."""
import numpy as np
import pytest

import synth
from tests.gpu_util import REL_TOL, oracle_value, rel_err, to_device

pytestmark = pytest.mark.gpu

BNS = (128, 112, 96, 80, 64, 48)
PAIR_WIDE = (256, 224)
WIDE_ONE_CTA = (160, 144)  # BF16x3 on one CTA (160: also the fused-split producer's wide tile)
PREC_CODE = {"tf32": 1, "3xtf32": 2, "bf16x3": 3}
TOL = {"bf16x3": REL_TOL, "3xtf32": 1e-5, "tf32": 1e-2}
# ragged M/N against 128-row (and 256-row CTA-pair) tiles and every N tile;
# K = 333 and 1100 end inside a k-block (zero-filled past K) and K = 1100
# takes two accumulator chunks in BF16x3
SHAPES = [(3, 300, 200, 333), (2, 520, 144, 1100), (4, 216, 776, 216)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_15080_b300 import build
    build.build()


def _gemm_lines(h):
    """batch, M, N, K, bn and the CTA-pair form of every GEMM launch of the
    lowered plan"""
    out = []
    for line in h.lowering_info().splitlines():
        f = line.split()
        if len(f) > 2 and f[2] == "gemm":
            d = {"pair": int("pair" in f)}
            for w in f:
                if "=" in w:
                    k, v = w.split("=", 1)
                    if k in ("batch", "M", "N", "K", "bn"):
                        d[k] = int(v)
            out.append(d)
    return out


@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "tf32"])
def test_every_orientation_and_n_tile(shape, prec, tmp_path):
    import torch
    from paper_2410_15080_b300 import from_network
    b, m, n, k = shape
    rng = np.random.default_rng(sum(shape))
    A = rng.uniform(-1, 1, (b, m, k))
    B = rng.uniform(-1, 1, (b, k, n))
    net = synth.HTN([synth.Tensor("QT", (0, 1, 3), A), synth.Tensor("QT", (0, 3, 2), B)], (0, 1, 2))
    ref = np.matmul(A, B).ravel()
    dev = to_device(net)
    seen = set()
    cases = [(sw, c, 0) for sw in (0, 1) for c in BNS]
    if prec == "bf16x3":  # one CTA's 160- and 144-column tiles; CTA pairs, with the two wider tiles only they have
        cases += [(sw, c, 0) for sw in (0, 1) for c in WIDE_ONE_CTA]
        cases += [(sw, c, 1) for sw in (0, 1) for c in BNS + PAIR_WIDE]
    for swap, bn, pair in cases:
        # the entry keyed both ways, so it applies whichever operand the
        # plan takes first (the other key's swap is the complement)
        path = tmp_path / f"t_{swap}_{bn}_{pair}.txt"
        p = PREC_CODE[prec]
        path.write_text(f"{p} {b} {m} {n} {k} : {swap} {bn} 0 0 0 {pair}\n"
                        f"{p} {b} {n} {m} {k} : {1 - swap} {bn} 0 0 0 {pair}\n")
        h = from_network(dev, net.output, prec=prec, autotune_table=str(path))
        g = _gemm_lines(h)
        assert len(g) == 1 and g[0]["bn"] == bn and g[0]["M"] == (n if swap else m), g
        assert g[0]["pair"] == pair, g
        out = h.contract()
        h.sync()
        torch.cuda.synchronize()
        err = rel_err(out.cpu().numpy(), ref)
        h.close()
        assert err <= TOL[prec], (swap, bn, pair, err)
        seen.add((swap, bn, pair))
    assert len(seen) == len(cases) == (32 if prec == "bf16x3" else 12)


def test_autotune_writes_a_table_the_plan_follows(tmp_path):
    """The mid-size ring (8 QTs of [64][144][144], 6 tensor-core steps):
    autotune its plan, re-plan with the table, contract, compare with the
    oracle."""
    import torch
    from paper_2410_15080_b300 import from_network
    net = synth.ring_htn()
    dev = to_device(net)
    path = tmp_path / "tiles.txt"
    h = from_network(dev, net.output, prec="bf16x3", autotune_table="")
    n = h.autotune(str(path), reps=3)
    h.close()
    assert n >= 1
    rows = {}
    for line in path.read_text().splitlines():
        if line.startswith("#"):
            continue
        key, val = line.split(":")
        kk = tuple(int(x) for x in key.split())
        sw, bn, ms, ms_rule, ms_base, pair = val.split()
        assert int(pair) in (0, 1) and int(bn) in BNS + (PAIR_WIDE if int(pair) else WIDE_ONE_CTA) \
            and int(sw) in (0, 1)
        # the padding rule's choice and the 128-column one are among those timed
        assert 0 < float(ms) <= min(float(ms_rule), float(ms_base))
        rows[kk] = (int(sw), int(bn), int(pair))
    assert len(rows) == n
    h2 = from_network(dev, net.output, prec="bf16x3", autotune_table=str(path))
    # every GEMM launch runs its problem's tuned choice (or is a fixed
    # 128- or 160-column producer of a fused split)
    for g in _gemm_lines(h2):
        match = [(sw, bn, pair) for (p, b, m, n_, k), (sw, bn, pair) in rows.items()
                 if p == 3 and b == g["batch"] and k == g["K"] and {m, n_} == {g["M"], g["N"]}
                 and g["M"] == (n_ if sw else m)]
        assert any(bn == g["bn"] and pair == g["pair"] for _, bn, pair in match) or \
            (g["bn"] in (128, 160) and g["pair"] == 0), (g, rows)
    out = h2.contract()
    h2.sync()
    torch.cuda.synchronize()
    err = rel_err(out.cpu().numpy(), oracle_value(net))
    h2.close()
    assert err <= REL_TOL


def test_summed_operand_pairs_on_cta_pairs(tmp_path):
    """A GEMM that sums four operand pairs in TMEM (the mid-size ring sliced
    over 16 wire-index values: the step that contracts a sliced index runs
    once per value of the other), forced onto CTA pairs by a tile table: the
    contraction matches the oracle."""
    import re
    import torch
    from paper_2410_15080_b300 import from_network
    net = synth.ring_htn()
    kw = dict(n_slices=16, slice_dim=4)
    dev = to_device(net)
    h = from_network(dev, net.output, prec="bf16x3", **kw)
    lines = [l for l in h.lowering_info().splitlines() if " gemm " in l]
    h.close()
    multi = [l for l in lines if re.search(r"runs=(\d+) launches=(\d+)", l).groups() == ("16", "4")]
    assert multi, lines
    g = {k: int(re.search(k + r"=(\d+)", multi[0]).group(1)) for k in ("batch", "M", "N", "K", "bn")}
    path = tmp_path / "pair.txt"
    path.write_text(f"3 {g['batch']} {g['M']} {g['N']} {g['K']} : 0 {g['bn']} 0 0 0 1\n"
                    f"3 {g['batch']} {g['N']} {g['M']} {g['K']} : 1 {g['bn']} 0 0 0 1\n")
    h = from_network(dev, net.output, prec="bf16x3", autotune_table=str(path), **kw)
    lines = [l for l in h.lowering_info().splitlines() if " gemm " in l]
    assert any(" pair " in l and "runs=16 launches=4" in l for l in lines), lines
    out = h.contract()
    h.sync()
    torch.cuda.synchronize()
    err = rel_err(out.cpu().numpy(), oracle_value(net))
    h.close()
    assert err <= REL_TOL
