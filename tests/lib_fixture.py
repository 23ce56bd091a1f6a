"""Build-once access to the CUDA library for tests (host-only calls work without a GPU)."""
import functools
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@functools.lru_cache(None)
def chol():
    sys.path.insert(0, ROOT)
    from paper_2409_14009_gb300 import build
    build.build()
    import paper_2409_14009_gb300 as P
    P.lib()
    return P
