"""CPU oracle of the neural visibility cache hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything here.  The
CUDA product path never imports, links or runs it, and it imports nothing
from the product package.
"""
from . import philox, nvc  # noqa: F401
