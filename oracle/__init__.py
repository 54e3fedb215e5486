"""FP64 CPU oracle of the metaball-DEM / LBM step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  See ``oracle/lbm_oracle.c``.
"""
from .oracle import Oracle, build, make_config, make_particle, mass_properties, particle_dict  # noqa: F401
