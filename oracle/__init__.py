"""CPU oracle (test infrastructure only; see seird_oracle's header)."""
from .seird_oracle import *  # noqa: F401,F403
