"""Gaussian lattice Boltzmann hot path on GB300 (sm_103a).

The compute path lives in the CUDA library ``libglbm.so`` (sources under
``csrc/``, C header ``include/glbm.h``); ``glbm`` is its Python binding.
"""
