"""FP64 CPU oracle (test infrastructure only; see ``lks_oracle`` for its scope and pins)."""
from .lks_oracle import *  # noqa: F401,F403
