"""B300-native (sm_103a) phaseless AFQMC hot path: a C-ABI CUDA library plus this thin binding."""
from ._lib import AfqmcError, Afqmc, PREC, draw_normals, load  # noqa: F401
