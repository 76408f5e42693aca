"""GB300 library for homomorphically encrypted convolution with Walsh-Hadamard
output-channel packing (Hyena, arXiv 2311.12519).

The compute path is libhyena.so (hand-written sm_103a CUDA + host C++); this
package only builds it (build.py) and binds its C ABI (hyena.py).  PyTorch,
where used by callers, provides device memory and streams.
"""
from . import build, hyena  # noqa: F401
