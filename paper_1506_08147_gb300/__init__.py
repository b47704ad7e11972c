"""GB300-native generation of DGDFT adaptive local basis functions.

The compute path is the CUDA shared library built from csrc/ (see build.py)
behind the C-ABI of include/dgdft_alb.h; ``binding`` marshals arguments to
it.  There is no CPU implementation in this package.
"""

from .binding import (  # noqa: F401
    DGDFT_PREC_FP64,
    DGDFT_PREC_MIXED,
    DGDFT_PRECOND_LEARNED,
    DGDFT_PRECOND_TETER,
    Context,
    DgdftError,
    element_dict,
    load,
    load_element,
)
