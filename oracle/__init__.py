"""CPU FP64 oracle (test infrastructure only; see dme_oracle's header)."""
from .dme_oracle import *  # noqa: F401,F403
from .dme_lowrank import *  # noqa: F401,F403
from .dme_leja import *  # noqa: F401,F403
