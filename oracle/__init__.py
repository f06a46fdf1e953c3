"""CPU FP64 oracle (test infrastructure only; see gpe_oracle's header)."""
from .gpe_oracle import *  # noqa: F401,F403
from .gpe_oracle import Problem, SolveOptions, pcg_solve  # noqa: F401
