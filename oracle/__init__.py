"""CPU oracle for the simplified MAME scheme (Huang, arXiv:2012.03525).

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports this package; only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg do.

Two independent implementations live here:

* ``acm_oracle.c`` -- plain FP64 C loops of Eqs. (2.10)-(2.11), the body
  force and the two-phase extension (Section 2), compiled with
  ``-O2 -ffp-contract=off`` and called through :mod:`oracle.c_oracle`;
* :mod:`oracle.ref_np` -- a NumPy restatement with ``np.roll`` (periodic
  grids only), used to cross-check the C loops on small grids;
* :mod:`oracle.conv_ref` -- the FP64 reference of the learned closure's
  convolution layers (forward and backward).
"""
