"""CPU oracle for the vertical secure-XGBoost Paillier hot path.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it. The product
path (``paper_2504_03909_b300``) never imports, links or runs anything here, and
this package imports nothing from the product path.

All arithmetic is plain Python integers (``pow`` is the modular exponentiation
library routine) or exact ``fractions.Fraction``; there is no blocking, fusion
or reordering beyond what the definitions state.
"""

from .paillier import *  # noqa: F401,F403
from . import tree  # noqa: F401
