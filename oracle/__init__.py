"""FP64 CPU oracle for the per-tile APIC reconstruction (WSI-APIC, Sec. 2.2-2.3).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
restatement of what the paper's reconstruction computes, written in numpy
float64/complex128 so that a reader can check each step against the paper's
equations by eye. Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product library (``paper_2407_20469_gb300``) never imports it and shares no
code, tables or constants with it.

Modules
-------
grid       Fourier-series conventions, pupil geometry, LED snapping, index sets
           (Eq. 1, Eq. 8, the U/P/Q regions of Eq. 11-13).
zernike    Noll-ordered, RMS-normalised Zernike polynomials (aberration basis).
forward    The forward model, Eq. 1-2 (simulated intensity stacks).
apic       The reconstruction: Kramers-Kronig recovery (Eq. 4-7), the
           phase-difference aberration solve (Eq. 8-10), correction and
           stitching, darkfield extension (Eq. 11-13) and the final inverse FFT.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test unless its docstring says "parity unpinned".
"""
