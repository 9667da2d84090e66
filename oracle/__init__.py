"""FP64 CPU oracle of the TPC sector tracker -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product path (paper_1910_12214_b300) never does.
"""
from .oracle import (OracleConfig, build_oracle, chi2, correct_clusters, fit_hits, propagate, run, trilinear)  # noqa: F401
