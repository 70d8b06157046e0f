"""GB300-native geometry-aware pairwise feature matching (arXiv 1512.06235, Sec. 6.2 and Appendix A).

The matching runs in ``libgeomatch.so`` (hand-written CUDA for sm_103a behind the C ABI of include/geomatch.h);
``geomatch`` is its ctypes binding.
"""
from .geomatch import (GM_PATH_AUTO, GM_PATH_MMA, GM_PATH_SIMT, GM_PATH_TC, Context, GeomatchError, GmPair,  # noqa
                       load_library, make_pair, split_matches)
