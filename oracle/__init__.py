"""CPU FP64 oracle (test infrastructure; see ``ytn_oracle`` for its scope and rules)."""
from .ytn_oracle import *  # noqa: F401,F403
from .ytn_oracle import FusionRecord  # noqa: F401
