"""CPU FP64 oracle of the PNGF DBS hot path (test infrastructure, not product)."""
from .pngf_oracle import *  # noqa: F401,F403
from .pngf_oracle import (BEST_IMPROVEMENT, COMBINE_MEAN, COMBINE_WORST, FIRST_IMPROVEMENT,  # noqa: F401
                          OBJ_MAX_WEIGHTED_POWER, OBJ_MIN_INSERTION_LOSS, DbsResult, Evaluation, Problem)
