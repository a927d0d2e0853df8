"""GB300-native spectral-bound graph coarsening (arXiv 2204.11757).

The compute path lives in the CUDA library ``libspcoarsen.so`` (sources in ``csrc/``); this
package holds its thin ctypes binding (``native``), the torch-facing API (``api``) and the
seeded synthetic workload generators (``inputs``).
"""
