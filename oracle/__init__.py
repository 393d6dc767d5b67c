"""Plain FP64 CPU oracle for the tunable-surface-tension pseudopotential LB method
(Li & Luo, arXiv 1306.6445).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it. The product
(the CUDA library and its Python binding) never imports, calls or links anything
here, and nothing here imports the product.

Modules
-------
lattice      the D2Q9 MRT pseudopotential update, step by step in the paper's order
             (Sec. II Eqs. 1-7, Eq. 8, Sec. IV Eqs. 17-19), vectorised over sites
             with numpy; periodic or bounce-back walls in y.
eos          equations of state, pseudopotentials, the critical point, the Maxwell
             construction, the mechanical-stability condition (Eq. 16) and the
             flat-interface surface tension that follows from Eq. 22.
diagnostics  Laplace-law measurement, interface height, capillary dispersion (Eq. 24).
bruteforce   an independent velocity-space twin of the update written with plain
             Python loops and explicit 9x9 matrices, for tiny lattices.

Parity status: every public function is pinned by a ``-m "not gpu"`` test except
the spurious-current magnitude (max |u| of a converged droplet), for which the
paper prints no value: parity unpinned.
"""
