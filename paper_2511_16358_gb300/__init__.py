"""GB300-native (sm_103a) iFCTN tensor completion: the PAM sweep of iFCTN-TC.

The compute path is libifctn.so (hand-written CUDA, C ABI in include/ifctn.h);
``paper_2511_16358_gb300.binding`` marshals arguments into it.  ``inputs``
holds seeded synthetic input generators.
"""
from . import inputs  # noqa: F401
