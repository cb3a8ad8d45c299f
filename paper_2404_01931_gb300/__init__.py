"""GB300-native FLIP step: CUDA kernels for sm_103a behind a C ABI (``include/flip.h``).

``paper_2404_01931_gb300.flip`` is the thin ctypes binding of the C ABI;
``paper_2404_01931_gb300.scenes`` generates the seeded synthetic inputs.
"""
__all__ = ["flip", "scenes"]
