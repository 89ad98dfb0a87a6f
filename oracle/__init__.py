"""CPU FP64 oracle of tensor-ring ALS (test infrastructure only; see trals_oracle)."""
from .trals_oracle import *  # noqa: F401,F403
