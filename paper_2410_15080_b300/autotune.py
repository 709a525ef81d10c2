"""Measure the GEMM tile table of this library's workloads on the local device.

    python -m paper_2410_15080_b300.autotune [--out PATH] [--reps N]
        [--workloads 100q,100q-free,mid] [--prec bf16x3] [--device 0]

Each workload is planned on a host-only handle (its shapes only, no tensor
data) exactly as the benchmark plans it, and qtpu_htn_autotune times every
valid orientation and N tile of each of its GEMM problems on synthetic
operands on the device, merging the fastest into the table.  By default the
table is gemm_tiles_b300.txt beside the library, which qtpu_htn_plan reads
when no other table is given."""
import argparse
import os

from .htn import HTN

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "gemm_tiles_b300.txt")


def workload_plans():
    """(network, plan options) of the benchmark's single-network workloads"""
    import synth
    big = dict(max_intermediate_bytes=8 << 30, n_candidates=256)
    return {"100q": (synth.ring_chords_htn(materialize=False), dict(big, n_slices=1024, slice_dim=4)),
            "100q-free": (synth.ring_chords_htn(materialize=False), big),
            "mid": (synth.ring_htn(), {})}


def tune(workloads, out=DEFAULT_TABLE, reps=5, prec="bf16x3", device=0) -> dict:
    plans = workload_plans()
    done = {}
    for name in workloads:
        net, kw = plans[name]
        h = HTN(device=-1)
        for t in net.tensors:
            h.add_tensor(t.inds, list(t.data.shape))
        h.set_output(net.output)
        h.plan(prec, autotune_table="", **kw)  # the padding rule's plan
        done[name] = h.autotune(out, reps=reps, device=device)
        h.close()
    return done


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--workloads", default="100q,100q-free,mid")
    ap.add_argument("--prec", default="bf16x3")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    for name, n in tune(a.workloads.split(","), a.out, a.reps, a.prec, a.device).items():
        print(f"{name}: {n} GEMM problems timed -> {a.out}")


if __name__ == "__main__":
    main()
