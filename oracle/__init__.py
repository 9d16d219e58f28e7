"""FP64 CPU oracle for the Keldysh loop bubble (test infrastructure only)."""
from .oracle import *  # noqa: F401,F403
