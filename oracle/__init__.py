"""FP64 CPU oracle for the CLOSURE hot path (arXiv 2403.09990).

TEST INFRASTRUCTURE ONLY.  A plain, slow restatement of what the GPU path
computes, written from the paper's definitions and algorithms in their order
and notation: the PURSE constraints (eq. 2, 3, 5), the distance to the
boundary (eq. 11), the boundary samplers (Alg. 2-5), RANSAG for 3D-3D
(Section IV, Step I), the centre statistics of Alg. 2, and the geodesic
gradient descent for the minimum enclosing geodesic ball (Section II,
Alg. 6 step rule), plus an exact Welzl ball used only as a pin.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never calls it and shares
no code with it.

Parity status per function is stated in each module header; a function that
no test pins to an independent fact says "parity unpinned".
"""
