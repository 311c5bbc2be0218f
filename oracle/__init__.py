"""Plain FP64 CPU oracle for the JGS2 per-vertex Jacobi sweep and its Gauss-Seidel mode
(test infrastructure only).

This package is the checker, not the product: only `tests/`, `__graft_entry__.smoke()` and
the CPU-baseline leg of `bench.py` may import it. It shares no code with the CUDA path;
the only common module is `scenes`, which builds seeded inputs and holds no arithmetic of
the method.

Every function states the passage of the paper (Lan et al., "JGS2: Near Second-order
Converging Jacobi/Gauss-Seidel for GPU Elastodynamics") it follows. Readings of passages
the paper leaves open are stated in the module docstrings (sweep.py, gs.py, contact.py,
cloth.py) and in the design notes.

Pins (tests/test_oracle_*.py): finite differences, rest-state closed forms, the
Schur-complement / KKT identities of Sec. 6, the optimality theorem of Sec. 4.2, rigid
rotation and translation invariance, the fixed point against a projected Newton solve,
the sweep counts of the convergence study (Sec. 8's rate is reached by the exact-subspace
sweep only), the Gauss-Seidel groups against the Jacobi path, the contact, friction and
cloth closed forms and finite differences. Parity is pinned for every function here except the cubature candidate draw, whose
random choices are compared by fit residual.
"""
