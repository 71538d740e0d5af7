"""GB300-native inverse matrix p-th root engine (Bini et al. iteration, arXiv:1703.02283).

The compute path lives in the C-ABI shared library built from ``csrc/``; ``pthroot`` is its thin
Python binding. ``workloads`` builds seeded synthetic inputs.
"""
