"""GB300 (sm_103a) solver for the simplified MAME scheme of Huang,
arXiv:2012.03525 -- a C-ABI CUDA library (``libacm.so``, include/acm.h) with a
thin Python binding (:mod:`paper_2012_03525_gb300.acm`)."""
