"""FP64 CPU oracle of the multi-mode difference-map iteration.

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never does.
"""
from . import dm  # noqa: F401
