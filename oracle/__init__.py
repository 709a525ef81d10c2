"""FP64 CPU oracle for hybrid tensor network (h-TN) contraction.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (``paper_2410_15080_b300``) and never
imports it; the only code both sides use is the seeded input generator
package ``synth``, which holds no contraction arithmetic.

Contents (each module cites the paper passage it restates):

* ``sim``      -- tiny density-matrix / statevector simulator (section 2.1
                  circuit knitting needs subcircuit expectation values).
* ``qpd``      -- the 6-term gate QPD of CZ and the 4x4 wire-cut tensor
                  (section 2.1, section 4.1 Eq. wire-tensor), Choi-matrix
                  identities, the naive knitting cost formula (section 2.1).
* ``knit``     -- the tiny 8-qubit cut circuit, its subcircuit tensors and the
                  brute-force knitting sum (Eq. knitting).
* ``tn``       -- the plain definition of tensor-network contraction with
                  hyper-indices (section 2.2), pairwise contraction in a
                  given order, brute force, and slicing.
* ``planner``  -- the reference greedy pairwise planner and slicer with exact
                  big-integer costs (section 4.2: cost depends on order).

Parity status of each function is stated in its module header; every function
here is pinned by a ``-m "not gpu"`` test against values the paper prints,
closed forms, invariants or brute force.
"""
