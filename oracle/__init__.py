"""CPU oracle for the strategy-annotated map/reduce hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import, call, link or run anything in this package. The
product library never routes through it, and it shares no code, header, table
or helper with the CUDA path.

Parts:

* ``patterns`` (c1): arrays as Python lists, the functional primitives of the
  paper's Fig. "Functional primitives" (map, reduce, zip, split, join, pair,
  fst, snd) plus the OpenCL-level annotations of Section 6 (mapGlobal,
  mapWorkgroup, mapLocal, mapSeq, toGlobal/toLocal/toPrivate, asVector,
  asScalar), all with their plain set-theoretic meaning (Section 5.1: an array
  of n elements is a function from {0..n-1}). Strategy expressions are built
  from these and evaluated element by element over a pluggable scalar
  arithmetic (binary32, int64, symbolic trees).
* ``loopnest`` (c2): the same strategy trees as plain single-threaded C loops
  (``loopnest.c``, built with ``-O2 -ffp-contract=off``), fast enough for the
  full-size workloads. Pinned to c1 bit for bit on tiny inputs.
* ``naive64`` (c3): exact / FP64 reference values (``math.fsum`` of exact
  products, numpy float64) used for error bounds.
* ``grads`` (c4): analytic adjoints in FP64 and central finite differences.

Functions whose result is fixed only by a tolerance (BF16 GEMM) are marked
"parity by tolerance" where they are defined; no function here is unpinned.
"""
