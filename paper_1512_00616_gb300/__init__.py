"""GB300 (sm_103a) implementation of the fully discrete periodic shooting and
periodic adjoint method (Zahr, Persson, Wilkening).  The compute path is the
C-ABI library libpp.so (include/pp.h); ``api`` is its thin Python binding."""
from . import api  # noqa: F401  (raises ImportError if libpp.so is not built)
