"""FP64 CPU oracle (test infrastructure only; see rihv_oracle's header)."""
from .rihv_oracle import *  # noqa: F401,F403
from .rihv_oracle import Optics  # noqa: F401
