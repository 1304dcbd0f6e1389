"""Plain FP64 CPU oracle of SAQ (arXiv 2509.12086) -- TEST INFRASTRUCTURE.

Only tests/, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import this package.  It shares no code with the CUDA library
(paper_2509_12086_gb300), and neither imports the other.
"""
from .saq_oracle import *  # noqa: F401,F403
