"""FP64 CPU oracle for separable dictionary learning (2D-OMP + TMOD).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
check of the package entry point and the CPU-baseline / reference legs of the
benchmark may import, call or execute anything in this package.  The CUDA
library never links, imports or calls it, and this package imports nothing
from the CUDA side: the two share no code.  Inputs come from the seeded
generators in ``paper_2007_03800_gb300.synth`` (data only, no method
arithmetic).
"""
from .sdl_oracle import *  # noqa: F401,F403
from . import denoise  # noqa: F401
from . import mlp  # noqa: F401
from . import ortho  # noqa: F401
from . import shortlist  # noqa: F401
from . import tmod3  # noqa: F401
