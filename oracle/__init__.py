"""FP64 CPU oracle for the per-scenario N-2 evaluation and the Risk Index.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code with the CUDA path (the only common
module is the seeded input generator ``paper_2512_08465_gb300.synth``, which
draws raw parameters and computes nothing of the method).

The oracle is deliberately plain: dense matrices, serial loops, the algorithm's
steps in the order the method states them, and outaged elements physically
*removed* from the network (the CUDA path masks them instead).

Module map (paper passages in parentheses):

* ``grid``      admittance matrices of the post-contingency network and the
                 island count by breadth-first search (Section II-B-3).
* ``opf``       primal-dual interior-point AC optimal power flow and the
                 operational-limit check (Section II-B-1).  The paper calls an
                 external OPF solver and does not state its algorithm; the
                 reading implemented is the MIPS primal-dual interior point
                 method (Wang, Murillo-Sanchez, Zimmerman, Thomas, 2007).
* ``dynamics``  linearised generator + voltage-regulator model at the OPF point,
                 Kron reduction to the generator internal nodes and the state
                 matrix A (Section II-B-2), derived by forward-mode automatic
                 differentiation of the plain state equations.
* ``eig``       balancing, Householder Hessenberg reduction and Francis
                 double-shift QR (plain C in ``eig.c``), eigenvalue statistics.
* ``pipeline``  one scenario end to end and the severity class (Sections II-A,
                 II-B).
* ``risk``      the Risk Index of Eq. 3 computed exactly with rationals.
* ``variants``  other backward-stable solves of the Newton systems (permuted LU,
                 Bunch-Kaufman LDL^T, refinement with exactly rounded residuals):
                 which scenarios' outcomes FP64 rounding decides.
* ``island``    main-island OPF of an islanded scenario with the reference
                 re-assigned, and its load shed (Sections II-A, V-A, VI: the
                 extension those passages point to).

Parity status per function is listed in each module header.
"""
