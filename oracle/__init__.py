"""FP64 CPU oracle for LAMP (arXiv 2511.11359).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py.  The product path never imports it.
"""
from .lamp_oracle import *  # noqa: F401,F403
