"""Python binding of the C ABI in ``include/qtpu_htn.h`` (argument marshalling only).

Every step of the contraction runs in ``libqtpu_htn.so``: this module passes
device pointers (``tensor.data_ptr()``), sizes and the current CUDA stream,
and turns status codes into exceptions.  There is no fallback: if the
library is missing, importing ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqtpu_htn.so")

QTPU_OK, QTPU_EINVAL, QTPU_ENOMEM, QTPU_ECUDA, QTPU_ESTATE, QTPU_ETIMEOUT, QTPU_ENOTSUP, QTPU_ELIMIT = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ESTATE", "ETIMEOUT", "ENOTSUP", "ELIMIT"]
QTPU_F32, QTPU_F64 = 0, 1
PREC = {"fp64": 0, "tf32": 1, "3xtf32": 2, "bf16x3": 3}
QTPU_QT, QTPU_CT = 0, 1

SYMBOLS = ["qtpu_htn_create", "qtpu_htn_add_tensor", "qtpu_htn_set_output", "qtpu_htn_plan",
           "qtpu_htn_plan_info", "qtpu_htn_autotune", "qtpu_htn_qpd_groups", "qtpu_htn_qpd_sample",
           "qtpu_htn_qpd_info", "qtpu_htn_num_tensors", "qtpu_htn_tensor_info", "qtpu_htn_knit_naive",
           "qtpu_qt_evaluate", "qtpu_htn_lowering_info", "qtpu_htn_output_size", "qtpu_htn_plan_stats",
           "qtpu_htn_exec_stats", "qtpu_htn_launch_features", "qtpu_htn_profile_launches", "qtpu_htn_contract",
           "qtpu_htn_contract_host", "qtpu_htn_contract_batch", "qtpu_htn_contract_batch_ex", "qtpu_htn_batch_info", "qtpu_htn_contract_slices", "qtpu_htn_sync", "qtpu_htn_selftest_timeout", "qtpu_htn_selftest_gemm_timeout", "qtpu_htn_destroy",
           "qtpu_htn_profile", "qtpu_htn_profile_read", "qtpu_pairwise_contract_noalloc",
           "qtpu_pairwise_noalloc_scratch_bytes", "qtpu_noalloc_status", "qtpu_noalloc_selftest_timeout",
           "qtpu_last_error",
           "qtpu_mlp_create", "qtpu_mlp_num_params", "qtpu_mlp_params", "qtpu_mlp_forward",
           "qtpu_mlp_gradients", "qtpu_mlp_train_step", "qtpu_mlp_destroy"]
KERNEL_CLASSES = ["contract", "split", "gemm", "reduce"]


class QtpuError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


class PlanOpts(C.Structure):
    _fields_ = [("max_intermediate_bytes", C.c_uint64), ("n_slices", C.c_uint32),
                ("slice_dim", C.c_uint32), ("prec", C.c_int), ("cost_model", C.c_int),
                ("seed", C.c_uint64), ("autotune_table", C.c_char_p), ("n_candidates", C.c_uint32),
                ("reuse_bytes", C.c_uint64), ("cost_model_path", C.c_char_p), ("search", C.c_uint32)]


class BatchOpts(C.Structure):
    _fields_ = [("persistent", C.c_int), ("wait_limit_ns", C.c_uint64), ("test_stall_network", C.c_int)]


_lib = None


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run python -m paper_2410_15080_b300.build")
        L = C.CDLL(LIB_PATH)
        vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
        L.qtpu_htn_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        L.qtpu_htn_add_tensor.argtypes = [vp, C.c_int, C.c_int, i64p, i64p, C.c_int, vp, i64p,
                                          C.POINTER(C.c_int)]
        L.qtpu_htn_set_output.argtypes = [vp, C.c_int, i64p]
        L.qtpu_htn_plan.argtypes = [vp, C.POINTER(PlanOpts)]
        L.qtpu_htn_plan_info.argtypes = [vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
        L.qtpu_htn_lowering_info.argtypes = [vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
        L.qtpu_htn_output_size.argtypes = [vp, i64p]
        L.qtpu_htn_plan_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.POINTER(C.c_uint64), i64p]
        L.qtpu_htn_exec_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_uint64), i64p]
        L.qtpu_htn_launch_features.argtypes = [vp, C.c_int, vp, i64p, C.POINTER(C.c_int)]
        L.qtpu_htn_profile_launches.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                                C.POINTER(C.c_int)]
        L.qtpu_htn_profile.argtypes = [vp, C.c_int]
        dp = C.POINTER(C.c_double)
        L.qtpu_htn_profile_read.argtypes = [vp, C.c_int, dp, i64p, dp, dp]
        L.qtpu_htn_contract.argtypes = [vp, vp]
        L.qtpu_htn_contract_host.argtypes = [vp, C.POINTER(vp), vp]
        L.qtpu_htn_contract_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), vp]
        L.qtpu_htn_contract_batch_ex.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), vp, C.POINTER(BatchOpts)]
        L.qtpu_htn_batch_info.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(C.c_int),
                                          C.POINTER(C.c_int)]
        L.qtpu_htn_contract_slices.argtypes = [vp, C.c_int64, C.c_int64, vp]
        L.qtpu_htn_sync.argtypes = [vp]
        L.qtpu_htn_selftest_timeout.argtypes = [vp, C.c_uint64]
        L.qtpu_htn_selftest_gemm_timeout.argtypes = [vp, C.c_int, C.c_uint64]
        L.qtpu_pairwise_contract_noalloc.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]
        L.qtpu_pairwise_noalloc_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
        L.qtpu_noalloc_status.argtypes = [vp]
        L.qtpu_noalloc_selftest_timeout.argtypes = [C.c_uint64, vp]
        L.qtpu_htn_destroy.argtypes = [vp]
        fp = C.POINTER(C.c_float)
        L.qtpu_mlp_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.c_int, C.c_int, C.c_uint64]
        L.qtpu_mlp_num_params.argtypes = [vp, i64p]
        L.qtpu_mlp_params.argtypes = [vp, vp, vp]
        L.qtpu_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
        L.qtpu_mlp_gradients.argtypes = [vp, vp, vp, C.c_int, vp, fp]
        L.qtpu_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, fp]
        L.qtpu_mlp_destroy.argtypes = [vp]
        L.qtpu_last_error.argtypes = [vp]
        L.qtpu_last_error.restype = C.c_char_p
        for s in SYMBOLS:
            if s != "qtpu_last_error":
                getattr(L, s).restype = C.c_int
        _lib = L
    return _lib


def _arr(vals, t=C.c_int64):
    vals = list(vals)
    return (t * max(1, len(vals)))(*vals)


class HTN:
    """One h-TN bound to a device and stream (device=-1: plan only)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._L = lib()
        self._h = C.c_void_p()
        if stream is None and device >= 0:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self._check(self._L.qtpu_htn_create(C.byref(self._h), device, C.c_void_p(stream or 0)), create=True)
        self.device = device
        self._keep = []  # tensors whose memory the library borrows
        self.n_tensors = 0

    def _check(self, st, create=False):
        if st != QTPU_OK:
            msg = self._L.qtpu_last_error(None if create else self._h).decode()
            raise QtpuError(st, msg)

    def add_tensor(self, inds: Sequence[int], dims: Sequence[int] = None, data=None, kind: int = QTPU_QT,
                   dtype: str | None = None, strides: Sequence[int] | None = None) -> int:
        """Register a tensor: ``data`` is a CUDA torch tensor (its shape and
        strides are used unless given) or None on a plan-only handle."""
        ptr = 0
        if data is not None:
            import torch
            assert data.device.type == "cuda", "tensors must be on the device"
            dims = list(data.shape) if dims is None else dims
            strides = list(data.stride()) if strides is None else strides
            dtype = {torch.float64: "f64", torch.float32: "f32"}[data.dtype]
            ptr = data.data_ptr()
            self._keep.append(data)
        dt = QTPU_F64 if (dtype or "f64") == "f64" else QTPU_F32
        tid = C.c_int(-1)
        self._check(self._L.qtpu_htn_add_tensor(
            self._h, kind, len(inds), _arr(inds), _arr(dims), dt, C.c_void_p(ptr),
            _arr(strides) if strides is not None else None, C.byref(tid)))
        self.n_tensors += 1
        return tid.value

    def set_output(self, inds: Sequence[int]):
        self._check(self._L.qtpu_htn_set_output(self._h, len(inds), _arr(inds)))
        self._out_inds = list(inds)

    def plan(self, prec: str = "bf16x3", max_intermediate_bytes: int = 0, n_slices: int = 0,
             slice_dim: int = 0, seed: int = 0, n_candidates: int = 0, reuse_bytes: int = 0,
             cost_model: int = 0, cost_model_path: str | None = None, autotune_table: str | None = None,
             search: int = 0):
        """autotune_table: GEMM tile table file (None: the measured table next
        to the library if present; "": the padding rule alone).  search: 0
        greedy, 1 hyper-search, 2 the exact tree alone."""
        o = PlanOpts(max_intermediate_bytes, n_slices, slice_dim, PREC[prec], cost_model, seed,
                     None if autotune_table is None else autotune_table.encode(), n_candidates,
                     reuse_bytes, cost_model_path.encode() if cost_model_path else None, search)
        self._check(self._L.qtpu_htn_plan(self._h, C.byref(o)))

    def autotune(self, table_path: str, reps: int = 5, device: int = -1) -> int:
        """Time every valid GEMM tile choice of the lowered plan on `device`
        (-1: the handle's) and merge the fastest per problem into
        `table_path`; returns the number of problems timed."""
        n = C.c_int(0)
        self._check(self._L.qtpu_htn_autotune(self._h, device, table_path.encode(), reps, C.byref(n)))
        return n.value

    def plan_info(self) -> str:
        need = C.c_size_t(0)
        self._check(self._L.qtpu_htn_plan_info(self._h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        self._check(self._L.qtpu_htn_plan_info(self._h, buf, need.value, None))
        return buf.value.decode()

    def lowering_info(self) -> str:
        need = C.c_size_t(0)
        self._check(self._L.qtpu_htn_lowering_info(self._h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        self._check(self._L.qtpu_htn_lowering_info(self._h, buf, need.value, None))
        return buf.value.decode()

    def output_size(self) -> int:
        n = C.c_int64()
        self._check(self._L.qtpu_htn_output_size(self._h, C.byref(n)))
        return n.value

    def plan_stats(self) -> dict:
        f, ns, nt, ws, nl = C.c_double(), C.c_int(), C.c_int(), C.c_uint64(), C.c_int64()
        self._check(self._L.qtpu_htn_plan_stats(self._h, C.byref(f), C.byref(ns), C.byref(nt), C.byref(ws),
                                                C.byref(nl)))
        return {"flops_total": f.value, "n_steps": ns.value, "n_tensor_core_steps": nt.value,
                "workspace_bytes": ws.value, "launches_per_contract": nl.value}

    def exec_stats(self) -> dict:
        """FLOPs one contract call executes (after slice reuse) and without
        reuse, kept bytes, kernel launches."""
        fe, fa, kb, nl = C.c_double(), C.c_double(), C.c_uint64(), C.c_int64()
        self._check(self._L.qtpu_htn_exec_stats(self._h, C.byref(fe), C.byref(fa), C.byref(kb), C.byref(nl)))
        return {"flops_executed": fe.value, "flops_all_slices": fa.value, "kept_bytes": kb.value,
                "launches": nl.value}

    def launch_features(self):
        """(features [n_launch, 32] float32, kernel launches per contraction of
        each) of the lowered launch list."""
        import numpy as np
        n = C.c_int(0)
        self._check(self._L.qtpu_htn_launch_features(self._h, 0, None, None, C.byref(n)))
        f = np.zeros((max(n.value, 1), 32), dtype=np.float32)
        cnt = np.zeros(max(n.value, 1), dtype=np.int64)
        self._check(self._L.qtpu_htn_launch_features(self._h, n.value, C.c_void_p(f.ctypes.data),
                                                     cnt.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(n)))
        return f[:n.value], cnt[:n.value]

    def profile_launches(self):
        """(launch index, ms) of every launch timed since the last read."""
        n = C.c_int(0)
        self._check(self._L.qtpu_htn_profile_launches(self._h, 0, None, None, C.byref(n)))
        cap = max(n.value, 1)
        idx = (C.c_int * cap)()
        ms = (C.c_double * cap)()
        self._check(self._L.qtpu_htn_profile_launches(self._h, cap, idx, ms, C.byref(n)))
        return list(idx)[:n.value], list(ms)[:n.value]

    def profile(self, enable: bool = True):
        self._check(self._L.qtpu_htn_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """Per kernel class: summed ms, launches, useful FLOPs, algorithmic bytes."""
        n = len(KERNEL_CLASSES)
        ms, fl, by = (C.c_double * n)(), (C.c_double * n)(), (C.c_double * n)()
        la = (C.c_int64 * n)()
        self._check(self._L.qtpu_htn_profile_read(self._h, n, ms, la, fl, by))
        return {k: {"ms": ms[i], "launches": la[i], "flops": fl[i], "bytes": by[i]}
                for i, k in enumerate(KERNEL_CLASSES)}

    def contract(self, out=None):
        """Enqueue the contraction; returns the FP64 output (device tensor)."""
        import torch
        if out is None:
            out = torch.empty(self.output_size(), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self._L.qtpu_htn_contract(self._h, C.c_void_p(out.data_ptr())))
        return out

    def contract_slices(self, first: int, count: int, out=None):
        """Sum of the results of slices [first, first + count) (device tensor)."""
        import torch
        if out is None:
            out = torch.empty(self.output_size(), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self._L.qtpu_htn_contract_slices(self._h, first, count, C.c_void_p(out.data_ptr())))
        return out

    def contract_host(self, host_arrays, out=None):
        """End-to-end form: host arrays in (one per tensor, in add order),
        host FP64 result out; copies happen inside the library call."""
        import numpy as np
        if out is None:
            out = np.empty(self.output_size(), dtype=np.float64)
        ptrs = (C.c_void_p * len(host_arrays))(*[a.ctypes.data if hasattr(a, "ctypes") else a.data_ptr()
                                                for a in host_arrays])
        self._check(self._L.qtpu_htn_contract_host(self._h, ptrs, C.c_void_p(out.ctypes.data)))
        return out

    def selftest_timeout(self, limit_ns: int):
        """Enqueue a bounded device wait that is bound to time out (see header)."""
        self._check(self._L.qtpu_htn_selftest_timeout(self._h, limit_ns))

    def selftest_gemm_timeout(self, pair: int, limit_ns: int):
        """Enqueue a GEMM launch whose waits are bound to time out (see header)."""
        self._check(self._L.qtpu_htn_selftest_gemm_timeout(self._h, int(pair), limit_ns))

    def sync(self):
        self._check(self._L.qtpu_htn_sync(self._h))

    def knit_naive(self, out=None):
        """Naive circuit knitting (Eq. knitting): the FP64 sum over every global
        instance; returns (output device tensor, number of instances)."""
        import torch
        n = 1
        for i in self._output_dims():
            n *= i
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=f"cuda:{self.device}")
        ni = C.c_double(0)
        self._check(self._L.qtpu_htn_knit_naive(self._h, C.c_void_p(out.data_ptr()), C.byref(ni)))
        return out, ni.value

    def _output_dims(self):
        if not hasattr(self, "_out_inds"):
            return []
        dims = {}
        for t in range(self.n_tensors):
            i = self.tensor_info(t)
            dims.update(zip(i["inds"], i["dims"]))
        return [dims[x] for x in self._out_inds]

    # ---- QPD sampling and h-TN simplification (section 4.3)
    def qpd_groups(self) -> int:
        """Number of gate-cut groups (rank-1 CTs between the same two QTs)."""
        n = C.c_int(0)
        self._check(self._L.qtpu_htn_qpd_groups(self._h, C.byref(n)))
        return n.value

    def qpd_sample(self, s_qpd: int, uniforms) -> "HTN":
        """The sampled, truncated network (unplanned, same output): uniforms is
        a CUDA float64 tensor of qpd_groups() * s_qpd values in [0, 1),
        group-major."""
        ptr = 0
        if uniforms is not None:
            import torch
            assert uniforms.device.type == "cuda" and uniforms.dtype == torch.float64 and uniforms.is_contiguous()
            assert uniforms.numel() >= self.qpd_groups() * s_qpd
            ptr = uniforms.data_ptr()
        out = C.c_void_p()
        self._check(self._L.qtpu_htn_qpd_sample(self._h, C.c_uint64(s_qpd), C.c_void_p(ptr), C.byref(out)))
        h = HTN.__new__(HTN)
        h._L, h._h, h.device = self._L, out, self.device
        h._out_inds = list(getattr(self, "_out_inds", []))
        h._keep = [self]  # the untouched tensors are borrowed from this network
        n = C.c_int(0)
        h._check(self._L.qtpu_htn_num_tensors(out, C.byref(n)))
        h.n_tensors = n.value
        return h

    def qpd_info(self):
        """[(fused length, values kept)] per group of a sampled network."""
        n = C.c_int(0)
        self._check(self._L.qtpu_htn_qpd_info(self._h, 0, None, None, C.byref(n)))
        a, b = (C.c_int64 * max(1, n.value))(), (C.c_int64 * max(1, n.value))()
        self._check(self._L.qtpu_htn_qpd_info(self._h, n.value, a, b, C.byref(n)))
        return [(a[i], b[i]) for i in range(n.value)]

    def tensor_info(self, t: int) -> dict:
        r = C.c_int(0)
        ids, dims, st = (C.c_int64 * 16)(), (C.c_int64 * 16)(), (C.c_int64 * 16)()
        dt, kd, ptr = C.c_int(0), C.c_int(0), C.c_void_p()
        self._check(self._L.qtpu_htn_tensor_info(self._h, t, 16, C.byref(r), ids, dims, st, C.byref(dt),
                                                 C.byref(kd), C.byref(ptr)))
        n = r.value
        return {"inds": tuple(ids[:n]), "dims": tuple(dims[:n]), "strides": tuple(st[:n]),
                "dtype": "f64" if dt.value == QTPU_F64 else "f32", "kind": kd.value, "ptr": ptr.value or 0}

    def tensor_view(self, t: int):
        """Tensor t as a CUDA torch tensor viewing the library's (or the
        caller's) device memory -- valid while this network lives."""
        import torch
        i = self.tensor_info(t)
        es = 8 if i["dtype"] == "f64" else 4

        class _View:
            __cuda_array_interface__ = {
                "shape": i["dims"], "typestr": "<f8" if es == 8 else "<f4", "data": (i["ptr"], False),
                "strides": tuple(x * es for x in i["strides"]), "version": 2}
        return torch.as_tensor(_View(), device=f"cuda:{self.device}")

    def close(self):
        if self._h:
            self._L.qtpu_htn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class QOp(C.Structure):
    _fields_ = [("kind", C.c_int), ("q0", C.c_int), ("q1", C.c_int), ("cut", C.c_int), ("side", C.c_int),
                ("u", C.c_double * 8)]


class QtProgram(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_ops", C.c_int), ("ops", C.POINTER(QOp)), ("n_cuts", C.c_int),
                ("cut_kind", C.POINTER(C.c_int)), ("cut_qubit", C.POINTER(C.c_int)), ("n_obs", C.c_int),
                ("paulis", C.c_char_p)]


QTPU_OP_U1, QTPU_OP_CZ, QTPU_OP_GATE_CUT = 0, 1, 2
QTPU_CUT_GATE, QTPU_CUT_MEASURE, QTPU_CUT_PREPARE = 0, 1, 2


def qt_evaluate(prog: dict, device: int = 0, stream: int | None = None):
    """The QT of one subcircuit program on the GPU (see qtpu_qt_evaluate):
    prog = {"n": qubits, "ops": [("u1", q, U) | ("cz", q0, q1) |
    ("gate_cut", q, cut, side)], "cuts": [("gate",) | ("measure", q) |
    ("prepare", q)], "paulis": [str per observable]}.  Returns a CUDA FP64
    tensor [observables, 6 or 4 per cut]."""
    import numpy as np
    import torch
    L = lib()
    ops = (QOp * max(1, len(prog["ops"])))()
    for i, op in enumerate(prog["ops"]):
        o = ops[i]
        if op[0] == "u1":
            o.kind, o.q0 = QTPU_OP_U1, op[1]
            U = np.asarray(op[2], dtype=np.complex128).ravel()
            for j in range(4):
                o.u[2 * j], o.u[2 * j + 1] = float(U[j].real), float(U[j].imag)
        elif op[0] == "cz":
            o.kind, o.q0, o.q1 = QTPU_OP_CZ, op[1], op[2]
        else:
            o.kind, o.q0, o.cut, o.side = QTPU_OP_GATE_CUT, op[1], op[2], op[3]
    kinds = {"gate": QTPU_CUT_GATE, "measure": QTPU_CUT_MEASURE, "prepare": QTPU_CUT_PREPARE}
    ck = _arr([kinds[c[0]] for c in prog["cuts"]], C.c_int)
    cq = _arr([c[1] if len(c) > 1 else -1 for c in prog["cuts"]], C.c_int)
    pa = "".join(prog["paulis"]).encode()
    p = QtProgram(prog["n"], len(prog["ops"]), ops, len(prog["cuts"]), ck, cq, len(prog["paulis"]), pa)
    dims = [6 if c[0] == "gate" else 4 for c in prog["cuts"]]
    out = torch.empty([len(prog["paulis"])] + dims, dtype=torch.float64, device=f"cuda:{device}")
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    ni = C.c_double(0)
    st = L.qtpu_qt_evaluate(device, C.c_void_p(stream), C.byref(p), C.c_void_p(out.data_ptr()), C.byref(ni))
    if st != QTPU_OK:
        raise QtpuError(st, L.qtpu_last_error(None).decode())
    return out


def contract_batch(htns: Sequence[HTN], outs, stream: int | None = None, persistent: bool | None = None,
                   wait_limit_ns: int = 0, test_stall_network: int = -1):
    """Contract many planned networks in one CUDA graph (see the C header).
    persistent: None = the library's choice (the persistent kernel when the
    small gather-only networks are at least half of the batch), True = always
    for them, False = graph branches only."""
    L = lib()
    hs = (C.c_void_p * len(htns))(*[h._h.value for h in htns])
    ps = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    o = BatchOpts(2 if persistent is None else (1 if persistent else 0), wait_limit_ns, test_stall_network)
    st = L.qtpu_htn_contract_batch_ex(hs, len(htns), ps, C.c_void_p(stream or 0), C.byref(o))
    if st != QTPU_OK:
        raise QtpuError(st, "contract_batch failed: " + htns[0]._L.qtpu_last_error(htns[0]._h).decode())


def batch_info(htns: Sequence[HTN], outs) -> dict:
    """Networks the persistent kernel contracts and its task count, for the
    most recent batch graph of these handles and outputs."""
    L = lib()
    hs = (C.c_void_p * len(htns))(*[h._h.value for h in htns])
    ps = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    npers, ntask = C.c_int(0), C.c_int(0)
    st = L.qtpu_htn_batch_info(hs, len(htns), ps, C.byref(npers), C.byref(ntask))
    if st != QTPU_OK:
        raise QtpuError(st, "no batch graph for these handles")
    return {"persistent_networks": npers.value, "tasks": ntask.value}


class MLP:
    """The cost model's perceptron through the C ABI (all arithmetic in the
    library's CUDA kernels; this class only marshals tensors)."""

    def __init__(self, in_dim: int, hidden: int = 256, seed: int = 1, device: int = 0, stream: int | None = None):
        import torch
        self._L = lib()
        self._m = C.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        st = self._L.qtpu_mlp_create(C.byref(self._m), device, C.c_void_p(stream or 0), in_dim, hidden, seed)
        if st != QTPU_OK:
            raise QtpuError(st, "qtpu_mlp_create failed")
        n = C.c_int64()
        self._L.qtpu_mlp_num_params(self._m, C.byref(n))
        self.n_params = n.value
        self.in_dim, self.hidden, self.device = in_dim, hidden, device

    def _ok(self, st, what):
        if st != QTPU_OK:
            raise QtpuError(st, what)

    def params(self, new=None):
        """FP32 master parameters as a numpy array (optionally set them first)."""
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        src = None
        if new is not None:
            new = np.ascontiguousarray(new, dtype=np.float32)
            src = C.c_void_p(new.ctypes.data)
        self._ok(self._L.qtpu_mlp_params(self._m, C.c_void_p(out.ctypes.data), src), "qtpu_mlp_params")
        return out

    def forward(self, x, out=None):
        import torch
        if out is None:
            out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self._ok(self._L.qtpu_mlp_forward(self._m, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(out.data_ptr())),
                 "qtpu_mlp_forward")
        return out

    def gradients(self, x, t):
        import numpy as np
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float()
        self._ok(self._L.qtpu_mlp_gradients(self._m, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0],
                                            C.c_void_p(g.ctypes.data), C.byref(loss)), "qtpu_mlp_gradients")
        return g, loss.value

    def train_step(self, x, t, lr: float = 1e-3) -> float:
        loss = C.c_float()
        self._ok(self._L.qtpu_mlp_train_step(self._m, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0],
                                             lr, C.byref(loss)), "qtpu_mlp_train_step")
        return loss.value

    def close(self):
        if self._m:
            self._L.qtpu_mlp_destroy(self._m)
            self._m = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pairwise_contract_noalloc(A, B, C_out, stream: int | None = None):
    """C_out[b] = A[b] @ B[b] through the allocation-free entry point (for
    callers that cannot allocate device memory at call time; see the C
    header).  A: [batch, M, K], B: [batch, K, N], C_out: [batch, M, N], all
    contiguous FP64 CUDA tensors owned by the caller."""
    import torch
    L = lib()
    b, m, k = A.shape
    n = B.shape[2]
    assert B.shape == (b, k, n) and C_out.shape == (b, m, n)
    for t in (A, B, C_out):
        assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
    if stream is None:
        stream = torch.cuda.current_stream(A.device).cuda_stream
    st = L.qtpu_pairwise_contract_noalloc(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                          C.c_void_p(C_out.data_ptr()), b, m, n, k, C.c_void_p(stream or 0))
    if st != QTPU_OK:
        raise QtpuError(st, L.qtpu_last_error(None).decode())
    return C_out


def noalloc_status(stream: int | None = None):
    """Wait for the stream and raise if an allocation-free call on the current
    device recorded a device-side failure (see qtpu_noalloc_status)."""
    L = lib()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = L.qtpu_noalloc_status(C.c_void_p(stream or 0))
    if st != QTPU_OK:
        raise QtpuError(st, L.qtpu_last_error(None).decode())


def noalloc_scratch_bytes(batch: int, m: int, n: int, k: int) -> int:
    """Exact scratch bytes the allocation-free call needs for these sizes."""
    L = lib()
    b = C.c_size_t(0)
    st = L.qtpu_pairwise_noalloc_scratch_bytes(batch, m, n, k, C.byref(b))
    if st != QTPU_OK:
        raise QtpuError(st, L.qtpu_last_error(None).decode())
    return b.value


def lowering_text(tensor_inds, dims: dict, output, prec="bf16x3", dtypes=None, **plan_kw) -> str:
    """Lower a plan on a host-only handle and return the launch list text."""
    h = HTN(device=-1)
    for t, inds in enumerate(tensor_inds):
        h.add_tensor(inds, [dims[i] for i in inds], dtype=(dtypes[t] if dtypes else "f64"))
    h.set_output(output)
    h.plan(prec, **plan_kw)
    t = h.lowering_info()
    h.close()
    return t


def plan_text(tensor_inds, dims: dict, output, max_intermediate_bytes=0, n_slices=0, slice_dim=0,
              seed=0, n_candidates=0) -> str:
    """Plan on a host-only handle and return the canonical plan text."""
    h = HTN(device=-1)
    for inds in tensor_inds:
        h.add_tensor(inds, [dims[i] for i in inds])
    h.set_output(output)
    h.plan("fp64", max_intermediate_bytes, n_slices, slice_dim, seed, n_candidates)
    t = h.plan_info()
    h.close()
    return t


def from_network(tensors, output, device: int = 0, prec: str = "bf16x3", stream: int | None = None,
                 **plan_kw) -> HTN:
    """Build and plan an HTN from (inds, device tensor, kind) triples."""
    h = HTN(device, stream)
    for t in tensors:
        inds, data = t[0], t[1]
        kind = t[2] if len(t) > 2 else QTPU_QT
        h.add_tensor(inds, data=data, kind=kind)
    h.set_output(output)
    h.plan(prec, **plan_kw)
    return h
