"""GB300 (sm_103a) Parareal for the 2.5D kinematic dynamo: the C-ABI library
libkd.so (include/kd.h) and its Python binding."""
from .kd import *  # noqa: F401,F403
from .kd import load, LIB_PATH, KdError, make_params, stats_dict  # noqa: F401
