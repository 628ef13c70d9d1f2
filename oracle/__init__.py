"""FP64 CPU oracle for the pseudo-spectral stochastic-PDE step (cuPSS, arXiv:2405.02410).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; the CUDA package never imports it.
"""
