"""GB300-native Pollock particle tracking (structured MODFLOW-style grids).

The compute path is the C-ABI library ``libmp.so`` (CUDA kernels for
sm_103a, declared in ``include/mp.h``); ``paper_2302_13590_gb300.mp`` is
the thin Python binding over it.  ``paper_2302_13590_gb300.inputs`` holds
the seeded synthetic field and release generators.
"""
