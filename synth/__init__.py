"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  This module only draws data; it holds none of the estimator's or
the inference algorithm's arithmetic."""
from .generators import *  # noqa: F401,F403
