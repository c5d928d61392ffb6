"""CPU FP64 oracle for the Monte Carlo NEGF walk path (Musland, Bergli, Flage-Larsen,
arXiv:1805.10164).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously correct restatement of what
the GPU path computes, written from the paper.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (``--impl reference`` and the ``cpu_baseline`` key) may import
it.  The product path (``paper_1805_10164_gb300``) never imports it and shares no code with it;
the two meet only in the seeded input generator, which holds none of the method's arithmetic.

Modules
-------
``wire``      square-lattice wire Hamiltonian, lead self-energies, dense G^r  (Sec. II.A, III.A)
``buttiker``  direct floating-probe solve of Eq. (buteq)                      (Sec. III.C)
``neumann``   the Neumann series of Eq. (iqof_t_el_db) with Buttiker Lambda   (Sec. II.E-F)
``markov``    Step 6' transition weights, injection (Step 4), exact absorption (Sec. II.D-F)
``alias``     Vose alias tables and their exact implied distribution          (Sec. III.B)
``philox``    Philox4x32-10 counter-based generator (Salmon et al., SC'11)
``walker``    the Step 6' random walk driven by Philox over integer alias tables
``current``   Fermi factors, lead current and its binomial standard error      (Sec. II.E, IV)
``adjoint``   FP64 derivatives of the transmission w.r.t. onsite energies and dephasing

Parity status of each function is stated in its docstring ("pinned by" or "parity unpinned").
"""
