"""FP64 CPU oracle (test infrastructure; never imported by the product path)."""
from .dmpt_oracle import *  # noqa: F401,F403
from . import dmpt_oracle  # noqa: F401
