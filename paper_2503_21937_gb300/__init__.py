"""GB300-native semi-naive fixpoint engine for semiring-tagged Datalog
(the hot path of Lobster, arXiv 2503.21937).

The compute lives in ``liblobster.so`` (hand-written sm_103a CUDA behind the C
ABI in ``include/lobster.h``); ``lobster`` is its ctypes binding.
"""
from .lobster import Engine, LobsterError, SEMIRINGS, load_library  # noqa: F401
