"""CPU oracle for the 1D sum-of-exponentials fast Gauss transform.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, link or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code, header, table or constant generator with the CUDA library.

Contents
--------
``soe_cf``      SOE construction (Sec. 2.3, eqs. 2.10-2.14; Sec. 3.3) from the
                Caratheodory-Fejer (CF) near-best rational approximation of
                e^z on the negative real axis, the E_n estimate of eq. 3.1, and
                the stabilised hyperbolic-contour SOE of Sec. 3.4 (eqs. 2.6-2.9).
``fgt_oracle.c``  plain FP64 C: O1 direct Gauss sum (eqs. 1.1-1.2),
                O2 direct SOE sum (eqs. 1.3, 4.1-4.2), O3 the paper's sorted
                forward/backward recurrences (eqs. 4.3-4.6), and the direct
                gradients of the Gauss and SOE transforms.
``oracle``      ctypes loader + numpy wrappers for ``fgt_oracle.c``.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(see ``tests/test_oracle_*.py``); none is "parity unpinned".
"""
