"""GB300 (sm_103a) implementation of the pseudo-spectral, semi-implicit
Euler-Maruyama step of stochastic PDEs on periodic lattices (cuPSS,
arXiv:2405.02410).  ``pss`` is the ctypes binding of libpss (include/pss.h);
``build`` compiles it."""
