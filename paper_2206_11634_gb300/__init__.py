"""GB300-native (sm_103a) lattice sweep of the coupled metaball-DEM / LBM method
(arXiv 2206.11634): node classification, fused stream/collide with
velocity-interpolated bounce-back, refilling, momentum-exchange force
reduction and the metaball DEM, behind the C ABI of include/lbm_metaball.h.
"""
from .lbm import (DEM_MODE, LIB_PATH, STORAGE, Batch, Lattice, LbmConfig, LbmError, LbmParticle,  # noqa: F401
                  load_library, make_config, make_particle, particle_dict)
