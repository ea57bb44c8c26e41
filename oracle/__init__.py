"""FP64 CPU oracle for the micropolar elastoplastic FFT-based solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may use it.

It restates the paper's method plainly, in float64, with no blocking, fusion
or reordering beyond what the paper's equations state:

* ``fft``           - its own mixed-radix FFT and a brute-force 3D DFT.
* ``constitutive``  - isotropic moduli (eq. stiffnesses_iso / elast_constitutive_iso),
                      equivalent stresses (eq. equiv_stress, equiv_couple_stress)
                      and the radial-return mapping of Algorithm 1.
* ``green``         - the reference medium's Green operator, written as the
                      per-wavevector solve of the Fourier-space balance laws
                      (eq. momemtum_balance) for the kinematics of eq. strains.
* ``solver``        - Algorithm 2 (basic scheme with time stepping) and the
                      error measures of eq. err, err_average, err_local.
* ``tangent``       - the continuum elastoplastic tangents of Appendix C.
* ``mnms``          - the numerically manufactured solution of Appendix D.1.

It shares no code with the CUDA library; both receive their inputs from the
``workloads`` package, which holds none of the method's arithmetic.
"""
