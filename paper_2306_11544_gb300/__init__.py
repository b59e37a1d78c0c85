"""GB300-native cell-mechanics step: voxel binning, neighbour-gather
repulsion/adhesion velocity and Adams-Bashforth-2 integration, as hand-written
sm_103a CUDA behind the C ABI of ``libmech`` (see ``include/mech.h``).

The binding (``paper_2306_11544_gb300.mech``) loads the compiled library on
first use; importing the package itself needs no GPU.
"""
__all__ = ["mech", "synth"]
