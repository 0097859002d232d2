"""CPU oracle for the Walsh -> boundary-wavelet change-of-basis products.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is written from the paper (Antun, "Recovering wavelet coefficients
from binary samples using fast transforms", arXiv 2106.00554) and from the
textbook definitions it relies on.  It is deliberately plain and slow:

* ``tables``   -- Daubechies filters, exact cell integrals of phi, restricted
                  Gram matrices, boundary (Cohen-Daubechies-Vial, "VMP")
                  scaling functions and boundary wavelets, computed in mpmath
                  at 60 significant digits and then rounded to float64.
* ``walsh``    -- Walsh functions straight from Def. 3.1 (bit by bit) and the
                  sequency-ordered Hadamard matrix of Sec. 3.1.
* ``wavelets`` -- the reconstruction bases on [0,1] of Sec. 3.2: the
                  cell-integral matrix T of the scaling basis B_{phi,j}, the
                  per-level synthesis matrices and the dense IDWT / DWT of
                  Remark 4.2.
* ``dense``    -- U = H_N T W^{-1} formed densely from the definition
                  U_{n,m} = <r_m, w_n> (Sec. 1.2 and the N x M section of
                  Sec. 4), in 1D and, one dimension at a time, in 2D.
* ``fast``     -- Algorithm 1 and Algorithm 2 as the paper states them (the
                  sum over l of D_l H_l of Sec. 4.1-4.2, Prop. 4.4 for the
                  edges) with a plain radix-2 FWHT.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against values the paper prints, closed forms, invariants or brute force.
The one partial pin is the VMP boundary space against Table 1 (the p = 2 row
agrees to 2e-3; the p >= 3 rows are not reproduced by the reading used here),
so for p >= 3 the VMP edges rest on their defining properties (orthonormality,
polynomial reproduction, staggered supports, nestedness) rather than on a
printed number.

The oracle shares no code with the CUDA library or its host planner; only the
seeded input generators (``paper_2106_00554_gb300.inputs``, which hold none of
the method's arithmetic) serve both.
"""
