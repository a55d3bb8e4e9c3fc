"""GB300 (sm_103a) binary-fluid D3Q19 lattice Boltzmann library.

The hot path -- phi stencil, fused f/g collision and streaming, FP64
conservation reductions -- runs in hand-written CUDA kernels behind the C ABI
of ``include/lb.h`` (``liblb.so``, built in-tree by ``build.build()``).
This package only marshals arguments to that library.
"""
from .nvbuild import build, library_path  # noqa: F401
from .lattice import KERNELS, PRECISIONS, VELOCITIES, Lattice, use_torch_allocator  # noqa: F401
from ._lib import LBError  # noqa: F401
from .batch import Batch  # noqa: F401
