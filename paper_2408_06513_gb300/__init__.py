"""GB300 (sm_103a) implementation of the de-cluttering iteration of Rave,
Molchanov and Linsen, "De-cluttering Scatterplots with Integral Images"
(arXiv 2408.06513), behind the C ABI of ``include/declutter.h``.

``paper_2408_06513_gb300.declutter`` is the ctypes binding; the kernels and
runtime live in ``csrc/`` and are built into ``libdeclutter.so`` by
``paper_2408_06513_gb300.build``.
"""

from . import declutter  # noqa: F401
from .declutter import *  # noqa: F401,F403
