"""FP64 CPU oracle of the FDTD-Bath step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg and reference
arm of ``bench.py`` may import this package (``__graft_entry__.build()`` compiles it).  It shares no code with the CUDA library:
``fdtd_oracle.c`` (time stepping, built by ``build.py``), ``oracle.py`` (ctypes
front end) and ``closed_forms.py`` (the paper's closed forms in numpy).
"""
