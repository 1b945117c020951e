"""FP64 CPU oracle of the NEP evaluation (test infrastructure only).

Only the tests, the smoke check and the timed CPU baseline import this package.
It shares no code with the CUDA library under paper_2603_01234_gb300/.
"""
from .oracle import *  # noqa: F401,F403
