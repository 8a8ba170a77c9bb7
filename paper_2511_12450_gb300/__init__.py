"""GB300-native layered-medium FMM boundary-integral solver (CUDA sm_103a behind a C ABI).

``paper_2511_12450_gb300.lfmm`` is the Python binding of include/lfmm.h; the
compiled library lives in ``paper_2511_12450_gb300/_lib`` and is built by
``paper_2511_12450_gb300._build.build()``.
"""

from . import lfmm  # noqa: F401
