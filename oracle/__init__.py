"""FP64 CPU oracle for AS-ICP grasp matching (arXiv 2412.08346).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA path (``paper_2412_08346_gb300``) never imports it and shares no code
with it; both sides only consume the arrays made by
``paper_2412_08346_gb300.synth``.

The arithmetic lives in ``asicp_oracle.c`` (plain C, float64, brute force,
compiled with ``-ffp-contract=off`` so it rounds the same on x86 and Arm);
this module builds it with gcc and wraps it with ctypes.
"""
from .oracle import (  # noqa: F401
    Oracle, build, rotation, rot_jacobian, nn, trilinear, gamma, bandwidth,
    stein_direction, fibonacci_init, quarter_init, select, centroid,
)
