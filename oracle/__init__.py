"""Oracle for finite-temperature orbital-free DFT (TEST INFRASTRUCTURE ONLY).

A plain, slow FP64 CPU implementation written from the paper (arXiv:1406.0835)
that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import it.  It shares no code with the CUDA
library and imports nothing from the package.
"""
from .ofdft_oracle import *  # noqa: F401,F403
