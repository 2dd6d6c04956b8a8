"""FP64 CPU oracle of the windowed beamspace MVDR hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it.  The product
path (the CUDA library and its Python binding) never calls it, and it shares
no code with that path: the two meet only in the seeded input generator of
``synth/``.

Every function follows a definition of the paper (section and equation
named in its docstring), in float64 / complex128, step by step and without
blocking or fusion.  A library primitive (numpy FFT, matrix product, linear
solve) is used where the definition is that primitive.

Parity pins (tests marked ``not gpu``) tie each function to something other
than itself: brute-force DFT sums, the closed-form Dirichlet kernel, the
Sherman-Morrison closed form for one interferer, the distortionless
constraint, the MVDR output-power identity, equality with full-dimensional
antenna-space MVDR when the window is the whole (unitary) beamspace, and
hand-computed fixtures in ``tests/golden``.
"""
from .beamspace_mvdr import *  # noqa: F401,F403
from .beamspace_mvdr import __all__  # noqa: F401
from . import learned_loading  # noqa: E402,F401
from . import range_doppler  # noqa: E402,F401
from . import upa  # noqa: E402,F401
from .abi import (oracle_apply, oracle_beamspace, oracle_channelize, oracle_mvdr_solve,  # noqa: E402,F401
                  oracle_pairs, oracle_window_cov)
