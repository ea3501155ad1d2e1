"""FP64 CPU oracle of the cross-spectrum FRB search -- TEST INFRASTRUCTURE ONLY.

Used by tests, the smoke check and the benchmark's CPU-baseline leg; never by the
library.  See ``reference.py`` for what each function computes and which passage
of the paper it follows.
"""
from . import reference  # noqa: F401
from ._clib import build  # noqa: F401
