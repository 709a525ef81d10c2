"""Seeded synthetic h-TN generators shared by the tests, the bench and the oracle.

This package holds input data only: index structure, dims, seeded random
entries, and the literal coefficient values a caller passes in as the
classical tensors.  It contains no contraction arithmetic and imports neither
the oracle nor the CUDA path.

A network is an ``HTN``: a list of ``Tensor(kind, inds, data)`` with ``data``
a numpy array whose axes follow ``inds``, plus the ``output`` index ids.
"""
from .networks import (  # noqa: F401
    HTN, Tensor, GATE_CT, WIRE_CT, ring_htn, ring_chords_htn, random_htn,
    random_batch, rank1_htn, rank1_qts_htn, tiny_random_htn,
)
