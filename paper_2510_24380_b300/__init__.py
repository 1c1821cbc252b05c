"""B300-native (sm_103a) exhaustive enumeration of combinatorial synthesis libraries (APEX hot path).

The CUDA library libapex_b300.so (C ABI in include/apex.h) does all the work; ``apex`` is the
ctypes binding. Build with ``python -m paper_2510_24380_b300.build``.
"""
from . import apex  # noqa: F401
from .apex import ApexError, Library, apex_count_compounds, apex_topk_select, load  # noqa: F401
