"""Plain FP64 CPU oracle for the FGA hot path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package. It never imports the product package and shares no code with it.
"""

from .fga_oracle import *  # noqa: F401,F403
from .fga_oracle import build  # noqa: F401
