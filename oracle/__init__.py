"""FP64 CPU oracle for SaCD (test infrastructure; see sacd_oracle.py)."""
from .sacd_oracle import *  # noqa: F401,F403
