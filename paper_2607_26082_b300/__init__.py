"""B300-native constrained DTT/FFT elasticity solver (Gelebart & Amouzou-Adoun,
"Constrained minimization problems and FFT-based solvers").

The compute path lives in libdtt.so (CUDA, sm_103a) behind the C ABI of include/dtt.h;
`paper_2607_26082_b300.dtt` is a thin ctypes binding with the same names, and
`paper_2607_26082_b300.rows` builds constraint rows (Sections 4.1-4.2) for it.
Importing this package does not load the library; `dtt.lib()` does, and raises if the
library is missing (there is no CPU fallback).
"""
__all__ = ["dtt", "rows"]
