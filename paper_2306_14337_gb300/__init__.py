"""GB300-native fixed-pattern KKT refactorization (arXiv 2306.14337).

The compute path is ``libkkt.so`` (hand-written CUDA for sm_103a behind the C
interface in ``include/kkt.h``); this package only marshals arguments.
"""
from ._capi import KKTError, load as load_library, lib_path
from .solver import KKTQueue, KKTSolver, kkt_solve

__all__ = ["KKTSolver", "KKTQueue", "kkt_solve", "KKTError", "load_library", "lib_path"]
