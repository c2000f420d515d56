"""GB300-native max-null permutation testing (NaivePT / RapidPT, arXiv 1703.01506).

The compute path lives in the C-ABI library ``lib/libpt.so`` (hand-written
sm_103a CUDA, declared in ``include/pt.h``); ``binding`` is its thin ctypes
front end with the same entry-point names. ``synth`` holds the seeded input
generators. Importing this package loads nothing; ``binding`` loads the
library on first use and raises if it has not been built.
"""

__all__ = ["binding", "synth"]
