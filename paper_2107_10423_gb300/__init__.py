"""GB300-native contour-deformation G0W0 (arXiv 2107.10423): CUDA library libgw.so behind a C ABI
(include/gw.h), a thin ctypes binding (``gw``) and seeded synthetic inputs (``synth``)."""
