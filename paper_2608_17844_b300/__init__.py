"""B300-native solver for regular finite arrays with a multilevel
block-Toeplitz Method of Moments matrix (arXiv 2608.17844): C-ABI library
libmoma (include/moma.h) and its thin Python binding.
"""
from .moma import *  # noqa: F401,F403
from .moma import EXPORTS, LIB_PATH, MomaError, lib  # noqa: F401
