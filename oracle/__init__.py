"""FP64 CPU oracle for the wavelet-adaptive ACM solver (Engels et al., arXiv:1912.05371).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference that the CUDA path is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. The product path (the C-ABI library
and its Python binding) never imports, links or calls anything here, and this package never
imports the product path. The two share no code; only the seeded input recipes in
``paper_1912_05371_gb300/workloads.py`` (which hold no arithmetic of the method) serve both.

Modules, each following the paper section it cites:

* ``forest``  -- blocks, octal treecodes, slots, neighbour tables            (Sec. 4.1, Sec. 3.5)
* ``mra``     -- DD-4 prediction, decimation, details, lifting              (Sec. 3.1-3.4)
* ``sync``    -- ghost-node values on the redundant block grid              (Sec. 4.2, Sec. 3.1)
* ``acm``     -- stencils, ACM right-hand side, RK4, time step, mask, force (Sec. 2.1-2.3)
* ``adapt``   -- refine-all / evolve / coarsen cycle, initial grid          (Sec. 3.5)
* ``adjoint`` -- discrete adjoint of RK4 steps on a frozen grid: gradients of a
                 force + energy objective w.r.t. the initial state and the sphere mask
                 (Sec. 2.1-2.3; the adjoint itself is an extension, not in the paper)
* ``plate``   -- moving rigid plate: box signed distance, stroke/pitch kinematics,
                 solid velocity, RK4 with the mask evaluated at every stage time (Sec. 2.2)
* ``checkpointing`` -- binomial checkpointing of the adjoint's reverse sweep (Griewank's
                 recursion, brute-force optimal splits; an extension, not in the paper)

Parity status: every function is pinned by a ``-m "not gpu"`` test against a closed form,
an invariant, a brute-force computation or a value the paper prints; none is "parity unpinned".
"""
