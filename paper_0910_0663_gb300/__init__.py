"""GB300 (sm_103a) implementation of the Virtual Transmission Method.

``paper_0910_0663_gb300.vtm`` is the user-facing API over the C ABI of
libvtm (``include/vtm.h``); ``workloads`` builds seeded synthetic circuits.
The CUDA library must be built (``paper_0910_0663_gb300.build.build()``)
before ``vtm`` can be imported.
"""
