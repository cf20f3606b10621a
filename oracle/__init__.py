"""CPU FP64 oracle (test infrastructure only; see qoc_oracle)."""
from .qoc_oracle import *  # noqa: F401,F403
from . import qoc_oracle  # noqa: F401
