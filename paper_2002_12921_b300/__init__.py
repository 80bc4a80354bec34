"""B300-native (sm_103a) hot path of the Vegas importance-sampling integrator.

The compute lives in the CUDA library built from ``csrc/`` (see ``build.py``)
behind the C ABI of ``include/vegas.h``; ``binding`` exposes the same calls to
Python.  ``workloads`` describes the seeded synthetic inputs.
"""
from .binding import *  # noqa: F401,F403
from .binding import Vegas, VegasError, lib  # noqa: F401
