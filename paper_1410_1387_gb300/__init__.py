"""GB300-native high-order finite-difference wave propagation.

The hot path (the radius-R stencil plus leapfrog step with fused source,
damping layer and receivers, isotropic and VTI) runs in hand-written sm_103a
CUDA kernels behind the C ABI declared in ``include/fd.h`` (``libfd.so``).
``paper_1410_1387_gb300.fd`` is the thin ctypes binding over that library;
``paper_1410_1387_gb300.synth`` draws the seeded synthetic inputs.
"""
__all__ = ["fd", "synth"]
