"""GB300 (sm_103a) implementation of the fully discrete periodic shooting and
periodic adjoint method (Zahr, Persson, Wilkening).  The compute path is the
C-ABI library libpp.so (include/pp.h); ``paper_1512_00616_gb300.api`` is its
thin Python binding and raises ImportError when libpp.so is not built (there is
no fallback).  ``paper_1512_00616_gb300.build`` compiles the library."""
