"""GB300-native even-odd Wilson-Dirac operator and CG solver (BSMBench hot
path).  The compute path is the CUDA library behind the C ABI declared in
include/bsm.h; `paper_1401_3733_gb300.bsm` is its thin ctypes binding and
raises at import when the library has not been built.  `fields` holds the
seeded synthetic inputs."""
