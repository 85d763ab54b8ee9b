"""GB300-native hot path of the Born-approximation method for hyperspectral diffuse optical
tomography (Saibaba, Kilmer, Miller & Fantini, arXiv:1410.0986): batched field solves,
Born rows, implicit J x / J^T y. The compute runs in libhydot.so (CUDA, sm_103a) behind
the C ABI in include/hydot.h; this package only marshals arguments.
"""
from ._lib import EXPORTS, HYDOT_FP64, HYDOT_MIXED, LIB_PATH, load  # noqa: F401
from .api import Context, HydotError, solve_batch  # noqa: F401
from .autograd import BornApply, born_apply  # noqa: F401
