"""Oracle for the NESA/EFIE path: a plain, slow, obviously correct FP64 CPU implementation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import, call or execute anything in this package.
The library (``paper_1801_03589_gb300``) shares no code with it and never imports it.

Modules (each function cites the part of the paper it follows):

* :mod:`oracle.quadrature`  triangle geometry and the 7-point degree-5 rule
* :mod:`oracle.rwg`         RWG basis functions on a triangle mesh (Sec. 2)
* :mod:`oracle.efie`        EFIE matrix rows: dense MoM and the near-field part (Eq. 1, Eq. 3)
* :mod:`oracle.tree`        octree, near lists and interaction lists (Sec. 2, Sec. 3)
* :mod:`oracle.nesa`        equivalent sources and the five far-field stages (Eqs. 4-7, 10-14)
* :mod:`oracle.rhs`         plane-wave excitation vector (Eq. 2, Eq. 3)
* :mod:`oracle.gmres`       restarted GMRES (Sec. 2, solver named there)
* :mod:`oracle.mie`         Mie series and far-field RCS of a PEC sphere (not in the paper)
* :mod:`oracle.nesa2d`      the 2D model problem of Sec. 3: log-kernel potential, quadtree
                            and its NESA product (Eqs. 8-14)

Pins (what each function is checked against) are the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``.  Parity unpinned: the absolute NESA accuracy at a given
number of equivalent sources (the paper prints no 3D figure for it).
"""
