"""CPU oracle for the KSG CMI estimator and the greedy network inference.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg are the only code allowed to import it.  The
product library (paper_1902_06828_gb300) never imports, links or calls it.
The oracle is independent of the CUDA path: it shares no code with it.
"""
from . import gauss, ksg, network  # noqa: F401
