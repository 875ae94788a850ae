"""GB300 (sm_103a) double-grid BSE Haydock library.

The compute path lives in the CUDA shared library built from `csrc/`; the
Python side (`bse.py`) only marshals arguments to its C ABI.  `synth` draws
the seeded model parameters.  Importing the package loads nothing native;
`paper_1602_01863_gb300.bse` loads the library on first use and raises if it
is missing.
"""
