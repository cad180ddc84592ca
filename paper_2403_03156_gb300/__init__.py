"""FSMP (arXiv 2403.03156) on GB300: per-waveform RJMCMC chains in hand-written sm_103a CUDA.

Importing the package loads nothing native. ``paper_2403_03156_gb300.fsmp`` is the Python
binding of the C-ABI library ``libfsmp.so`` (built by ``paper_2403_03156_gb300.build``);
``paper_2403_03156_gb300.workloads`` generates seeded synthetic inputs.
"""
