"""GB300-native Keldysh loop bubble (KeldyshQFT, arXiv:2405.20996): CUDA kernels for
sm_103a behind the C ABI of include/kb.h, with a ctypes binding (kb) and a small
PyTorch-facing helper (engine)."""

from . import kb  # noqa: F401
