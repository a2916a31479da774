"""FP64 CPU oracle of the local BIE / walk-on-spheres DtN method.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The product path (paper_1210_1491_gb300) never
imports it, and it never imports the product path.
"""
from .oracle import *  # noqa: F401,F403
