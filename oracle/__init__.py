"""CPU oracle for the homomorphic vital-sign chain -- TEST INFRASTRUCTURE.

This package is a plain, slow, obviously-correct restatement of the RNS-CKKS
evaluator and of the paper's kernel chain (Sec. "Cloud-Side Algorithms",
kernels K1-K7; Table 1 depth accounting; Table 7 scheme parameters).  It
exists only to check the CUDA library: the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` are the only code allowed to import
it.  It shares no code with the CUDA path; the two meet only through the
seeded input generators in ``synth`` and through documented data formats
(coefficient-form residue arrays).

Modules
-------
_native   ctypes loader of ``core.c`` (128-bit modular arithmetic, NTT)
params    deterministic prime selection, HE-standard bound, size arithmetic
ckks      encoding, key generation, encryption and every evaluator operation
circuits  slot layout, public constants and the two circuits (FIR+DFT, vital)
plain     the FP64 plaintext pipeline of the same formulas

Functions whose result has no independent pin say "parity unpinned" in their
docstring; at present there are none.
"""
