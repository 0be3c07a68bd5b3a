"""FP64 CPU oracle of the wave path tracer (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library.
"""
from .oracle import Oracle, build, philox4x32_10, cone_dir, fresnel_dielectric, ggx_eval, ggx_sample, frame, half_to_double  # noqa: F401
