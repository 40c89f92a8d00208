"""FP64 CPU oracle for mixed-state rPIE with Adam position refinement.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is a plain, slow, obviously-correct restatement of the method of
Guzzi et al., "A modular software framework for the design and
implementation of ptychography algorithms" (arXiv 2205.04295):

* ``model``        -- thin-sample exit wave, far-field propagation, mixed-state
                      intensities (Background section, Eqs. 1-3; M-rPIE
                      section, Eq. 4).
* ``grouping``     -- rounding of scan positions to crop boxes and the greedy
                      partition into pairwise-disjoint groups (the build's
                      schedule; the paper itself is sequential).
* ``rpie``         -- one M-rPIE iteration: modulus constraint (Eq. 7),
                      probe update (Eq. 5), object update (Eq. 6), optional
                      XCORR_A registration + Adam position step.
* ``registration`` -- subpixel cross-correlation registration by an upsampled
                      matrix DFT (Adam-based position refinement section,
                      after Guizar-Sicairos et al., Opt. Lett. 33, 2008).
* ``adam``         -- Adam as a per-position gain controller (Algorithm 1,
                      Eqs. 8-9; Kingma & Ba Algorithm 1).
* ``grad``         -- amplitude loss of the bilinear-crop forward model and
                      its analytic gradient (differentiable form).
* ``modes``        -- orthogonalisation of the probe modes through the
                      eigendecomposition of their Gram matrix (mixed state
                      of Eq. 4, after Thibault & Menzel 2013).

Everything is complex128 / float64.  Library primitives used as steps:
``numpy.fft`` (the DFT), ``numpy.matmul`` (matrix DFT) and
``numpy.linalg.eigh`` (Hermitian eigendecomposition).  The oracle shares
no code with the CUDA library and never imports it.
"""
