"""GB300-native FDiRW hot path (Mao, Hu & Li, "A GPU accelerated mixed-precision FDiRW solver").

Every cell of a porous, strongly inhomogeneous domain launches a unit mass; an explicit 7-point FD
diffusion is marched over a local window for one macro step to give that source's spreading kernel
(Sec. 3.1), and the field advances by the superposition c'(x) = sum_s c(s) P(s -> x) (Eq. 8).

* ``fdirw``  -- ctypes binding of libfdirw.so (C ABI in include/fdirw.h); all compute is CUDA (sm_103a).
* ``build``  -- compiles libfdirw.so in-tree with nvcc.
* ``synth``  -- seeded synthetic microstructures, diffusivity maps and initial fields.
"""
from . import synth  # noqa: F401
from .fdirw import (FDiRW, FDiRWBatch, FDiRWCoarse, FdirwError, Net, PRECISIONS, fdirw_create,  # noqa: F401
                    fdirw_create_batch, fdirw_create_coarse, fdirw_read_coarse, fdirw_destroy, fdirw_get_info, fdirw_kernels, fdirw_last_error, fdirw_mass, fdirw_read_kernels,
                    fdirw_read_radius, fdirw_set_velocity, fdirw_stable_dt, fdirw_step)

__all__ = ["FDiRW", "FDiRWBatch", "FDiRWCoarse", "FdirwError", "Net", "PRECISIONS", "fdirw_create", "fdirw_create_batch",
           "fdirw_create_coarse", "fdirw_read_coarse", "fdirw_destroy", "fdirw_get_info", "fdirw_kernels", "fdirw_last_error", "fdirw_mass", "fdirw_read_kernels",
           "fdirw_read_radius", "fdirw_set_velocity", "fdirw_stable_dt", "fdirw_step", "synth"]
