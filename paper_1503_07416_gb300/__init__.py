"""GB300 (sm_103a) FAS multigrid implicit time step for the hydrodynamic PFC
and CDFT freezing models (Baskaran, Guan, Lowengrub), behind the C ABI of
include/fm.h.  ``fm`` is the ctypes binding; ``build`` compiles libfm.so."""
