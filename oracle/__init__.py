"""Plain, slow, FP64 CPU oracle for the multi-resolution fast lattice Green's
function (FLGF) method (Dorschner, Yu, Mengaldo & Colonius, arXiv:1911.10228).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library under
``paper_1911_10228_gb300/csrc`` and never reads anything that library writes.

Modules
-------
lgf       LGF values: 1-D Bessel integral (Eq. GL_B) by fixed panel quadrature
          with an analytic tail, far-field expansions A^2 and A^3 (Sec. 2),
          and the table/asymptotic switch.
conv      The plain definitions: brute-force discrete convolution
          (Eq. discretConv), whole-domain zero-padded FFT convolution, and the
          7-point Laplacian L_Q.
flgf      The uniform FLGF method on one resolution (Sec. 2.1): octree,
          near/influence lists, Lagrange interpolation J and anterpolation
          R = J^T, block-wise zero-padded FFT convolution, upward pass,
          level interaction, downward pass.
multires  The block-refined scheme (Sec. 3): coarsening C, two-FMM
          leaf/non-leaf subtraction, coarse-fine interpolation J^l, source
          correction, accumulation.

Parity status of each function is stated in its module header.
"""
