"""Independent FP64 CPU reference of the correlator path (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package; the product library never does.  The C core is in
`wick_oracle.c`, the operator tables in `operators.py`.

Parity status: every function is pinned by the not-gpu tests (closed forms,
invariances, brute force on tiny inputs, exact modular identities); none is
"parity unpinned".
"""
