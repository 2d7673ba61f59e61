"""CPU FP64 oracle of the PNGF DBS hot path (test infrastructure, not product)."""
from .pngf_oracle import *  # noqa: F401,F403
from .pngf_oracle import (BEST_IMPROVEMENT, FIRST_IMPROVEMENT, OBJ_MAX_WEIGHTED_POWER,  # noqa: F401
                          OBJ_MIN_INSERTION_LOSS, DbsResult, Evaluation, Problem)
